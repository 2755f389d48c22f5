// Fused layer-pair kernels for 1-D bases (one translation unit per basis
// dimension, compiled in parallel).
#include "sv_pair.cuh"

namespace disk {
DISK_PAIR_INSTANTIATE(1)
}  // namespace disk
