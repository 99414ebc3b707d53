// complex128 instantiation of the row-local combinations with a fused sparse product
#include "kr_rowsp_launch.cuh"
namespace kr {
KR_INSTANTIATE_ROWSP(double)
}
