// Instantiations of the spatially varying layer kernel for 2-D bases.
#include "sv_layer.cuh"

namespace disk {
DISK_SV_INSTANTIATE(2, false)
}  // namespace disk
