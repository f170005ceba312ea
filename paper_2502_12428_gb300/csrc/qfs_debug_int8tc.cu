// Parity hook kernels of the int8 tensor-core form (one quartic, every intermediate array written out).
#include "qfs_kernels.cuh"
namespace qfs {
QFS_DEFINE_DEBUG_LAUNCHER(2)
}
