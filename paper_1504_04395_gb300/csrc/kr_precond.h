// ILU(0) right preconditioning (kr_precond.cu).
#pragma once

#include <cuda_runtime.h>

namespace kr {

struct Operator;

// Factorise the operator's CSR values (FP64, host) and upload L, U, U^H, L^H with their level
// schedules into op.ilu.  Returns a kr_status: KR_OK, KR_BAD_ARG (a missing diagonal entry or
// a duplicate entry), KR_BREAKDOWN (a zero pivot).
int build_ilu0(Operator& op);

// Y = M^{-1} V (adjoint = false) or M^{-H} V (adjoint = true) for n x s complex128 blocks; tmp is
// an n x s scratch block (Y may equal V, not tmp).
void apply_ilu0(const Operator& op, bool adjoint, int s, const double2* V, double2* Y, double2* tmp,
                cudaStream_t st);

}  // namespace kr
