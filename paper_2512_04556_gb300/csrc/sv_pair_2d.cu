// Fused layer-pair kernels for 2-D bases (one translation unit per basis
// dimension, compiled in parallel).
#include "sv_pair.cuh"

namespace disk {
DISK_PAIR_INSTANTIATE(2)
}  // namespace disk
