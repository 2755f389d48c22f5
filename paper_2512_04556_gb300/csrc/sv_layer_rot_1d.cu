// Instantiations of the rotated spatially varying layer kernel for 1-D bases.
#include "sv_layer.cuh"

namespace disk {
DISK_SV_INSTANTIATE(1, true)
}  // namespace disk
