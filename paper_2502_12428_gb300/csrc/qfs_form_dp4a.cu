// dp4a form: the power chain runs as 4-way int8 dot products (IDP4A) with int32 accumulation on CUDA cores.
#include "qfs_kernels.cuh"
namespace qfs {
QFS_DEFINE_FORM_LAUNCHER(1)
}
