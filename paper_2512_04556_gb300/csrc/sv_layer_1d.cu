// Instantiations of the spatially varying layer kernel for 1-D bases.
#include "sv_layer.cuh"

namespace disk {
DISK_SV_INSTANTIATE(1, false)
}  // namespace disk
