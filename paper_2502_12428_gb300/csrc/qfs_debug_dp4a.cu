// Parity hook kernels of the dp4a form (one quartic, every intermediate array written out).
#include "qfs_kernels.cuh"
namespace qfs {
QFS_DEFINE_DEBUG_LAUNCHER(1)
}
