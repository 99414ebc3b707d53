// complex64 instantiation of the row-local linear combinations
#include "kr_rows_launch.cuh"
namespace kr {
KR_INSTANTIATE_LIN(float)
}
