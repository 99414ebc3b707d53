// complex64 instantiation of the row kernels
#include "kr_rows_launch.cuh"
namespace kr {
KR_INSTANTIATE_ROWS(float)
}
