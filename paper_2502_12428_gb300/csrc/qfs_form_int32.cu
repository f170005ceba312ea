// int32 form: every multiply-add of the power chain is an IMAD on CUDA cores.
#include "qfs_kernels.cuh"
namespace qfs {
QFS_DEFINE_FORM_LAUNCHER(0)
}
