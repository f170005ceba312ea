// int8 tensor-core form: the power chain runs as mma.sync m16n8k32 u8 contractions with int32 accumulation.
#include "qfs_kernels.cuh"
namespace qfs {
QFS_DEFINE_FORM_LAUNCHER(2)
}
