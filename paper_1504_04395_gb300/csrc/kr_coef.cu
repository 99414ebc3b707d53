// Coefficient phases: the small FP64 steps between the row kernels of each method.
//
// Each phase runs as one CTA.  It reads reduced Gram / trace / norm values
// (red), updates the device solver state, and writes the scalar or s x s
// coefficients that the next row kernel applies.  A phase that detects
// convergence, divergence, a non-finite value or a breakdown sets the state's
// done flag, after which every later kernel of the solve returns at once.
#include "kr_engine.h"
#include "kr_profile.h"
#include "kr_small.cuh"

namespace kr {
using namespace small;

namespace {

enum : int { ST_OK = 0, ST_BREAKDOWN = 1, ST_DIVERGED = 2, ST_NAN = 3, ST_MAXIT = 4 };
// fields of the per-column Li-QMR state (slot SL_TMP5, field f of column c at f * s + c)
enum : int {
  LQ_RHO = 0, LQ_XI, LQ_T, LQ_DELTA, LQ_DELTAP, LQ_ROT1C, LQ_ROT1S, LQ_ROT2C, LQ_ROT2S, LQ_RHON, LQ_XIN
};

__device__ __forceinline__ double2* SLP(const CoefArgs& a, int i) { return a.ar + (size_t)i * kSlotElems; }

__device__ __forceinline__ void fail(DevState* st, int status) {
  __syncthreads();
  if (threadIdx.x == 0 && !st->done) {
    st->status = status;
    st->done = 1;
  }
  __syncthreads();
}
__device__ __forceinline__ bool is_done(const DevState* st) {
  __syncthreads();
  const bool d = *(volatile const int*)&st->done != 0;
  __syncthreads();
  return d;
}

// Stopping test after one iteration (relative residual rnorm / ||R_0||).
__device__ void monitor(const CoefArgs& a, double rnorm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    DevState* st = a.st;
    st->iter += 1;
    const double rel = rnorm / st->res0;
    st->rel = rel;
    a.hist[st->iter] = rel;
    if (rel < st->best) { st->best = rel; st->best_iter = st->iter; }
    if (!isfinite(rel)) { st->status = ST_NAN; st->done = 1; }
    else if (rel <= st->tol) { st->status = ST_OK; st->done = 1; }
    else if (rel > 1e8) { st->status = ST_DIVERGED; st->done = 1; }
    else if (st->iter >= st->maxit) { st->status = ST_MAXIT; st->done = 1; }
    else if (st->stall > 0 && rel > 1.0 && st->iter - st->best_iter >= max(st->stall, st->best_iter)) {
      st->status = ST_MAXIT;  // above the starting residual and no new minimum for a while
      st->done = 1;
    }
  }
  __syncthreads();
}

// num / den with the scalar breakdown rule; returns status (0 ok)
__device__ int check_div(double2 num, double2 den, double2* out) {
  if (!finite2(num) || !finite2(den)) return ST_NAN;
  const double ad = cabsd(den);
  if (ad == 0.0 || ad <= kEps * cabsd(num)) return ST_BREAKDOWN;
  *out = cdiv(num, den);
  return ST_OK;
}

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 neg(double2 a) { return make_double2(-a.x, -a.y); }

// copy reduced slots into an arena slot
__device__ __forceinline__ void from_red(double2* dst, const double2* red, int cnt) { copy(dst, red, cnt); }

// complex Givens rotation G = [[c, s], [-conj(s), c]] (c real) with G [a; b] = [r; 0]
__device__ void givens(double2 a, double2 b, double* c, double2* s, double2* r) {
  if (b.x == 0.0 && b.y == 0.0) { *c = 1.0; *s = make_double2(0.0, 0.0); *r = a; return; }
  if (a.x == 0.0 && a.y == 0.0) { *c = 0.0; *s = make_double2(1.0, 0.0); *r = b; return; }
  const double aa = cabsd(a), ab = cabsd(b);
  const double nu = hypot(aa, ab);
  const double2 ph = make_double2(a.x / aa, a.y / aa);
  *c = aa / nu;
  const double2 t = cm(ph, cj(b));
  *s = make_double2(t.x / nu, t.y / nu);
  *r = make_double2(ph.x * nu, ph.y * nu);
}

__device__ void stack2(double2* dst, const double2* top, const double2* bot, int s) {  // [top; bot] (2s x s)
  for (int i = threadIdx.x; i < 2 * s * s; i += blockDim.x) dst[i] = (i < s * s) ? top[i] : bot[i - s * s];
  __syncthreads();
}
__device__ void split2(double2* top, double2* bot, const double2* src, int s) {
  for (int i = threadIdx.x; i < 2 * s * s; i += blockDim.x) {
    if (i < s * s) top[i] = src[i]; else bot[i - s * s] = src[i];
  }
  __syncthreads();
}
__device__ void scale_mat(double2* dst, const double2* src, double2 f, int cnt) {
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) dst[i] = cm(f, src[i]);
  __syncthreads();
}

__device__ double trace_prod(const double2* A, const double2* B, int s, bool adjA, double* scratch, double* im_out) {
  // tr(op(A) B) with op(A) = A^H when adjA; returns real part, imaginary part in *im_out
  double re = 0.0, im = 0.0;
  for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
    const int i = idx / s, j = idx % s;  // term op(A)[i][j] * B[j][i]
    double2 aij = adjA ? cj(A[j * s + i]) : A[i * s + j];
    const double2 p = cm(aij, B[j * s + i]);
    re += p.x;
    im += p.y;
  }
  for (int off = 16; off >= 1; off >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, off);
    im += __shfl_down_sync(0xffffffffu, im, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { scratch[2 * warp] = re; scratch[2 * warp + 1] = im; }
  __syncthreads();
  double tr = 0.0, ti = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tr += scratch[2 * w]; ti += scratch[2 * w + 1]; }
  __syncthreads();
  *im_out = ti;
  return tr;
}

}  // namespace

__global__ void __launch_bounds__(256) coef_kernel(CoefArgs a) {
  __shared__ double scratch[64];
  __shared__ int iscr[4];
  __shared__ double2 hv[2 * kMaxS];
  DevState* st = a.st;
  if (*(volatile const int*)&st->done) return;
  const int s = a.s;
  const int ss = s * s;
  const double2* red = a.red;

  switch (a.phase) {
    case PH_INIT: {
      if (threadIdx.x == 0) {
        const double r = sqrt(red[a.i0].x);
        st->res0 = r;
        st->iter = 0;
        a.hist[0] = 1.0;
        if (!isfinite(r)) { st->status = ST_NAN; st->done = 1; }
        else if (r == 0.0) { st->status = ST_OK; st->done = 1; }
        else if (st->maxit <= 0) { st->status = ST_MAXIT; st->done = 1; }
      }
      break;
    }
    case PH_MONITOR: {
      monitor(a, sqrt(red[a.i0].x));
      break;
    }
    case PH_FILL_ONES: {
      fill(SLP(a, SL_ONES), ss, make_double2(1.0 / s, 0.0));
      break;
    }
    // ------------------------------------------------------------ scalar BiCG (Alg. 2, 4)
    case PH_SC_RHO0: {
      if (threadIdx.x == 0) st->sc_rho = red[a.i0];
      break;
    }
    case PH_SC_ALPHA: {
      if (threadIdx.x == 0) {
        double2 al;
        const int r = check_div(st->sc_rho, red[a.i0], &al);
        if (r) { st->status = r; st->done = 1; } else SLP(a, SL_ALPHA)[0] = al;
      }
      break;
    }
    case PH_SC_ALPHA_CONJ: {  // alpha = rho / conj(red): the denominator's reduction came conjugated
      if (threadIdx.x == 0) {
        double2 al;
        const double2 d = make_double2(red[a.i0].x, -red[a.i0].y);
        const int r = check_div(st->sc_rho, d, &al);
        if (r) { st->status = r; st->done = 1; } else SLP(a, SL_ALPHA)[0] = al;
      }
      break;
    }
    case PH_SC_BETA: {
      monitor(a, sqrt(red[a.i1].x));
      if (is_done(st)) break;
      if (threadIdx.x == 0) {
        double2 be;
        const double2 rn = red[a.i0];
        const int r = check_div(rn, st->sc_rho, &be);
        if (r) { st->status = r; st->done = 1; } else { SLP(a, SL_BETA)[0] = be; st->sc_rho = rn; }
      }
      break;
    }
    // ------------------------------------------------------------ Li-BiCG (Alg. 1)
    case PH_LI_RHO0: {
      copy(SLP(a, SL_TMP5), red + a.i0, s);
      break;
    }
    case PH_LI_ALPHA: {
      if (threadIdx.x == 0) {
        for (int c = 0; c < s; ++c) {
          double2 al;
          const int r = check_div(SLP(a, SL_TMP5)[c], red[a.i0 + c], &al);
          if (r) { st->status = r; st->done = 1; break; }
          SLP(a, SL_ALPHA)[c] = al;
        }
      }
      break;
    }
    case PH_LI_BETA: {
      monitor(a, sqrt(red[a.i1].x));
      if (is_done(st)) break;
      if (threadIdx.x == 0) {
        for (int c = 0; c < s; ++c) {
          double2 be;
          const int r = check_div(red[a.i0 + c], SLP(a, SL_TMP5)[c], &be);
          if (r) { st->status = r; st->done = 1; break; }
          SLP(a, SL_BETA)[c] = be;
        }
        if (!st->done)
          for (int c = 0; c < s; ++c) SLP(a, SL_TMP5)[c] = red[a.i0 + c];
      }
      break;
    }
    // ------------------------------------------------------------ Li-BiCGStab (columnwise)
    case PH_LS_ALPHA: {  // i0: rt_c^H v_c
      if (threadIdx.x == 0) {
        for (int c = 0; c < s; ++c) {
          double2 al;
          const int r = check_div(SLP(a, SL_TMP5)[c], red[a.i0 + c], &al);
          if (r) { st->status = r; st->done = 1; break; }
          SLP(a, SL_ALPHA)[c] = al;
        }
      }
      break;
    }
    case PH_LS_OMEGA: {  // i0: s_c^H t_c (conjugated: t_c^H s_c), i1: t_c^H t_c
      if (threadIdx.x == 0) {
        for (int c = 0; c < s; ++c) {
          const double2 ts = cj(red[a.i0 + c]);
          const double tt = red[a.i1 + c].x;
          if (!finite2(ts) || !isfinite(tt)) { st->status = ST_NAN; st->done = 1; break; }
          const double2 om = tt == 0.0 ? make_double2(0.0, 0.0) : make_double2(ts.x / tt, ts.y / tt);
          SLP(a, SL_OMEGA)[c] = om;
          SLP(a, SL_NOMEGA)[c] = neg(om);
        }
      }
      break;
    }
    case PH_LS_BETA: {  // i0: rt_c^H r_c (new), i1: ||R||^2
      monitor(a, sqrt(red[a.i1].x));
      if (is_done(st)) break;
      if (threadIdx.x == 0) {
        for (int c = 0; c < s; ++c) {
          double2 b1, b2;
          int r = check_div(red[a.i0 + c], SLP(a, SL_TMP5)[c], &b1);
          if (!r) r = check_div(SLP(a, SL_ALPHA)[c], SLP(a, SL_OMEGA)[c], &b2);
          if (r) { st->status = r; st->done = 1; break; }
          const double2 be = cm(b1, b2);
          SLP(a, SL_BETA)[c] = be;
          SLP(a, SL_GAMMA)[c] = neg(cm(be, SLP(a, SL_OMEGA)[c]));
        }
        if (!st->done)
          for (int c = 0; c < s; ++c) SLP(a, SL_TMP5)[c] = red[a.i0 + c];
      }
      break;
    }
    // ------------------------------------------------------------ Bl-BiCG (Alg. 3)
    case PH_BL_G0: {
      from_red(SLP(a, SL_G), red + a.i0, ss);
      break;
    }
    case PH_BL_ALPHA:
    case PH_RQ_ALPHA: {
      double2 *T0 = SLP(a, SL_TMP0), *G = SLP(a, SL_G);
      copy(T0, red + a.i0, ss);
      copy(SLP(a, SL_ALPHA), G, ss);
      if (!lu_solve(T0, SLP(a, SL_ALPHA), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      adjoint(T0, red + a.i0, s);
      adjoint(SLP(a, SL_ALPHAH), G, s);
      if (!lu_solve(T0, SLP(a, SL_ALPHAH), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      if (a.phase == PH_RQ_ALPHA) matmul(SLP(a, SL_AC), SLP(a, SL_ALPHA), SLP(a, SL_C), s, s, s);
      break;
    }
    case PH_BL_BETA: {
      monitor(a, sqrt(red[a.i1].x));
      if (is_done(st)) break;
      double2 *T0 = SLP(a, SL_TMP0), *T1 = SLP(a, SL_TMP1), *G = SLP(a, SL_G);
      copy(T1, red + a.i0, ss);
      copy(T0, G, ss);
      copy(SLP(a, SL_BETA), T1, ss);
      if (!lu_solve(T0, SLP(a, SL_BETA), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      adjoint(T0, G, s);
      adjoint(SLP(a, SL_BETAH), T1, s);
      if (!lu_solve(T0, SLP(a, SL_BETAH), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      copy(G, T1, ss);
      break;
    }
    // ------------------------------------------------------------ CholQR2 (thin QR, Eq. (QR))
    case PH_QR1: {  // i0 Gram of Z, i1 -> R1, i2 -> R1^{-1}, x0 = n
      double2 *R1 = SLP(a, a.i1), *R1i = SLP(a, a.i2);
      copy(R1, red + a.i0, ss);
      if (!chol_upper(R1, s, iscr)) {
        // shifted Cholesky: G + sigma I, sigma = 11 (n s + s (s + 1)) eps ||G||_F
        const double nrm = fro(red + a.i0, ss, scratch);
        const double sigma = 11.0 * (a.x0 * s + s * (s + 1.0)) * kEps * nrm;
        copy(R1, red + a.i0, ss);
        for (int i = threadIdx.x; i < s; i += blockDim.x) R1[i * s + i].x += sigma;
        __syncthreads();
        if (!chol_upper(R1, s, iscr)) { fail(st, ST_BREAKDOWN); break; }
      }
      tri_inv_upper(R1i, R1, s);
      break;
    }
    case PH_QR2: {  // i0 Gram of Z R1^{-1}, i1 R1, i2 -> R2^{-1}, i3 -> S = R2 R1
      double2* T0 = SLP(a, SL_TMP0);
      copy(T0, red + a.i0, ss);
      if (!chol_upper(T0, s, iscr)) { fail(st, ST_BREAKDOWN); break; }
      tri_inv_upper(SLP(a, a.i2), T0, s);
      matmul(SLP(a, a.i3), T0, SLP(a, a.i1), s, s, s);
      break;
    }
    // ------------------------------------------------------------ Bl-BiCG-rQ (Alg. 5)
    case PH_RQ_INIT: {
      from_red(SLP(a, SL_G), red + a.i0, ss);
      break;
    }
    case PH_RQ_C: {
      double2* T0 = SLP(a, SL_TMP0);
      matmul(T0, SLP(a, SL_S), SLP(a, SL_C), s, s, s);
      copy(SLP(a, SL_C), T0, ss);
      matmul(T0, SLP(a, SL_SH), SLP(a, SL_CH), s, s, s);
      copy(SLP(a, SL_CH), T0, ss);
      const double nc = fro(SLP(a, SL_C), ss, scratch);
      monitor(a, nc);
      break;
    }
    case PH_RQ_BETA: {
      double2 *T0 = SLP(a, SL_TMP0), *T1 = SLP(a, SL_TMP1), *T2 = SLP(a, SL_TMP2), *T3 = SLP(a, SL_TMP3);
      double2* G = SLP(a, SL_G);
      copy(T1, red + a.i0, ss);                         // G_new = Qh_new^H Q_new
      matmul(SLP(a, SL_BETA), SLP(a, SL_SH), T1, s, s, s, true, false);  // Sh^H G_new
      copy(T0, G, ss);
      if (!lu_solve(T0, SLP(a, SL_BETA), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      adjoint(T3, T1, s);                               // G_new^H
      matmul(SLP(a, SL_BETAH), SLP(a, SL_S), T3, s, s, s, true, false);  // S^H G_new^H
      adjoint(T0, G, s);
      if (!lu_solve(T0, SLP(a, SL_BETAH), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      (void)T2;
      copy(G, T1, ss);
      break;
    }
    // ------------------------------------------------------------ Gl-BiCGStab
    case PH_GS_ALPHA: {
      if (threadIdx.x == 0) {
        double2 al;
        const int r = check_div(st->sc_rho, red[a.i0], &al);
        if (r) { st->status = r; st->done = 1; } else SLP(a, SL_ALPHA)[0] = al;
      }
      break;
    }
    case PH_GS_OMEGA:
    case PH_BS_OMEGA: {  // i0 tr(S^H T), i1 ||T||^2, i2 (Bl) Rt^H T
      if (threadIdx.x == 0) {
        const double2 ts = cj(red[a.i0]);  // tr(T^H S)
        const double2 tt = make_double2(red[a.i1].x, 0.0);
        if (!finite2(ts) || !finite2(tt)) { st->status = ST_NAN; st->done = 1; }
        else {
          const double2 om = (tt.x == 0.0) ? make_double2(0.0, 0.0) : cdiv(ts, tt);
          SLP(a, SL_OMEGA)[0] = om;
          SLP(a, SL_NOMEGA)[0] = neg(om);
        }
      }
      if (a.phase == PH_BS_OMEGA) copy(SLP(a, SL_RTT), red + a.i2, ss);
      break;
    }
    case PH_GS_BETA: {
      monitor(a, sqrt(red[a.i1].x));
      if (is_done(st)) break;
      if (threadIdx.x == 0) {
        double2 b1, b2;
        const double2 rn = red[a.i0];
        int r = check_div(rn, st->sc_rho, &b1);
        if (!r) r = check_div(SLP(a, SL_ALPHA)[0], SLP(a, SL_OMEGA)[0], &b2);
        if (r) { st->status = r; st->done = 1; }
        else {
          const double2 be = cm(b1, b2);
          SLP(a, SL_BETA)[0] = be;
          SLP(a, SL_GAMMA)[0] = neg(cm(be, SLP(a, SL_OMEGA)[0]));
          st->sc_rho = rn;
        }
      }
      break;
    }
    // ------------------------------------------------------------ Bl-BiCGStab
    case PH_BS_G0:
    case PH_BSR_INIT: {
      from_red(SLP(a, SL_G), red + a.i0, ss);
      break;
    }
    case PH_BS_ALPHA:
    case PH_BSR_ALPHA: {
      double2* T0 = SLP(a, SL_TMP0);
      copy(SLP(a, SL_M), red + a.i0, ss);
      copy(T0, red + a.i0, ss);
      copy(SLP(a, SL_ALPHA), SLP(a, SL_G), ss);
      if (!lu_solve(T0, SLP(a, SL_ALPHA), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      break;
    }
    case PH_BS_BETA: {  // i0 Rt^H R_new, i1 ||R_new||^2
      monitor(a, sqrt(red[a.i1].x));
      if (is_done(st)) break;
      double2* T0 = SLP(a, SL_TMP0);
      copy(T0, SLP(a, SL_M), ss);
      scale_mat(SLP(a, SL_BETA), SLP(a, SL_RTT), make_double2(-1.0, 0.0), ss);
      if (!lu_solve(T0, SLP(a, SL_BETA), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      scale_mat(SLP(a, SL_B2), SLP(a, SL_BETA), SLP(a, SL_NOMEGA)[0], ss);  // -omega beta
      copy(SLP(a, SL_G), red + a.i0, ss);
      break;
    }
    // ------------------------------------------------------------ Bl-BiCGStab-rQ
    case PH_BSR_OMEGA: {  // i0 Sp^H Tp, i1 Tp^H Tp, i2 Rt^H Tp
      double2 *T0 = SLP(a, SL_TMP0), *C = SLP(a, SL_C);
      matmul(T0, C, C, s, s, s, false, true);  // C C^H
      double im1, im2;
      // tr(Tp^H Sp C C^H) with Tp^H Sp = (Sp^H Tp)^H
      const double nr = trace_prod(red + a.i0, T0, s, true, scratch, &im1);
      const double dr = trace_prod(red + a.i1, T0, s, false, scratch, &im2);
      const double2 num = make_double2(nr, im1), den = make_double2(dr, im2);
      if (!finite2(num) || !finite2(den)) { fail(st, ST_NAN); break; }
      const double2 om = (den.x == 0.0 && den.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(num, den);
      if (threadIdx.x == 0) { SLP(a, SL_OMEGA)[0] = om; SLP(a, SL_NOMEGA)[0] = neg(om); }
      copy(SLP(a, SL_RTT), red + a.i2, ss);
      matmul(SLP(a, SL_AC), SLP(a, SL_ALPHA), C, s, s, s);
      scale_mat(SLP(a, SL_OC), C, om, ss);
      break;
    }
    case PH_BSR_C: {  // i0 Rt^H Q_new; Sigma in SL_S
      double2 *T0 = SLP(a, SL_TMP0), *T1 = SLP(a, SL_TMP1), *C = SLP(a, SL_C), *Sg = SLP(a, SL_S);
      matmul(T0, Sg, C, s, s, s);
      copy(C, T0, ss);
      monitor(a, fro(C, ss, scratch));
      if (is_done(st)) break;
      copy(T0, SLP(a, SL_M), ss);
      scale_mat(SLP(a, SL_BETA), SLP(a, SL_RTT), make_double2(-1.0, 0.0), ss);
      if (!lu_solve(T0, SLP(a, SL_BETA), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      const double nS = fro(Sg, ss, scratch);
      bool bad = false;
      for (int i = 0; i < s; ++i) bad = bad || cabsd(Sg[i * s + i]) <= 64.0 * kEps * nS;
      if (bad) { fail(st, ST_BREAKDOWN); break; }
      tri_inv_upper(T1, Sg, s);
      matmul(SLP(a, SL_B2), SLP(a, SL_BETA), T1, s, s, s);
      scale_mat(SLP(a, SL_B3), SLP(a, SL_B2), SLP(a, SL_NOMEGA)[0], ss);
      copy(SLP(a, SL_G), red + a.i0, ss);
      break;
    }
    // ------------------------------------------------------------ Gl-QMR / eGl-QMR
    case PH_QMR_INIT: {  // i0 ||R0||^2, i1 ||W-start||^2 (for econ: of the n-vector)
      if (threadIdx.x == 0) {
        const double rho = sqrt(red[a.i0].x);
        double xi = sqrt(red[a.i1].x);
        if (st->econ) xi *= sqrt((double)s);
        if (xi == 0.0 || !isfinite(xi)) { st->status = xi == 0.0 ? ST_BREAKDOWN : ST_NAN; st->done = 1; }
        st->rho_k = rho;
        st->xi_k = xi;
        st->t = make_double2(rho, 0.0);
        st->k = 0;
        st->have_rot1 = st->have_rot2 = 0;
        SLP(a, SL_INVRHO)[0] = make_double2(1.0 / rho, 0.0);
        SLP(a, SL_INVXI)[0] = make_double2(1.0 / xi, 0.0);
      }
      break;
    }
    case PH_QMR_DELTA: {
      if (threadIdx.x == 0) { st->delta = red[a.i0]; st->delta_prev = make_double2(0.0, 0.0); }
      break;
    }
    case PH_QMR_COEF1: {  // i0 tr(W^H Y)
      if (threadIdx.x == 0) {
        const double2 d = st->delta;
        if (!finite2(d)) { st->status = ST_NAN; st->done = 1; }
        else if (d.x == 0.0 && d.y == 0.0) { st->status = ST_BREAKDOWN; st->done = 1; }
        else {
          st->k += 1;
          const double2 al = cdiv(red[a.i0], d);
          double2 be = make_double2(0.0, 0.0), ga = make_double2(0.0, 0.0);
          if (st->k >= 2) {
            const double2 q = cdiv(d, st->delta_prev);
            be = make_double2(st->xi_k * q.x, st->xi_k * q.y);
            ga = cj(make_double2(st->rho_k * q.x, st->rho_k * q.y));
          }
          SLP(a, SL_ALPHA)[0] = al;
          SLP(a, SL_BETA)[0] = be;
          SLP(a, SL_GAMMA)[0] = ga;
        }
      }
      break;
    }
    case PH_QMR_COEF2: {  // i0 ||Vt||^2, i1 ||Wt||^2, i2 tr(Wt^H Vt)
      if (threadIdx.x == 0) {
        const double rn = sqrt(red[a.i0].x);
        double xn = sqrt(red[a.i1].x);
        if (st->econ) xn *= sqrt((double)s);
        double2 u2 = make_double2(0.0, 0.0), u1 = SLP(a, SL_BETA)[0], u0 = SLP(a, SL_ALPHA)[0];
        if (st->have_rot2) {
          const double c = st->rot2_c.x;
          const double2 sn = st->rot2_s;
          u2 = cm(sn, u1);
          u1 = make_double2(c * u1.x, c * u1.y);
        }
        if (st->have_rot1) {
          const double c = st->rot1_c.x;
          const double2 sn = st->rot1_s;
          const double2 n1 = make_double2(c * u1.x + cm(sn, u0).x, c * u1.y + cm(sn, u0).y);
          const double2 n0 = make_double2(-cm(cj(sn), u1).x + c * u0.x, -cm(cj(sn), u1).y + c * u0.y);
          u1 = n1;
          u0 = n0;
        }
        double c;
        double2 sn, ukk;
        givens(u0, make_double2(rn, 0.0), &c, &sn, &ukk);
        if (!finite2(ukk) || !isfinite(rn) || !isfinite(xn)) { st->status = ST_NAN; st->done = 1; }
        else if (ukk.x == 0.0 && ukk.y == 0.0) { st->status = ST_BREAKDOWN; st->done = 1; }
        else {
          const double2 tau = make_double2(c * st->t.x, c * st->t.y);
          st->t = neg(cm(cj(sn), st->t));
          const double2 iu = cdiv(make_double2(1.0, 0.0), ukk);
          SLP(a, SL_CV)[0] = iu;
          SLP(a, SL_CD2)[0] = neg(cm(u2, iu));
          SLP(a, SL_CD1)[0] = neg(cm(u1, iu));
          SLP(a, SL_TAU)[0] = tau;
          SLP(a, SL_NTAU)[0] = neg(tau);
          st->rot2_c = st->rot1_c;
          st->rot2_s = st->rot1_s;
          st->have_rot2 = st->have_rot1;
          st->rot1_c = make_double2(c, 0.0);
          st->rot1_s = sn;
          st->have_rot1 = 1;
          st->rho_n = rn;
          st->xi_n = xn;
          SLP(a, SL_INVRHO)[0] = make_double2(rn > 0.0 ? 1.0 / rn : 0.0, 0.0);
          SLP(a, SL_INVXI)[0] = make_double2(xn > 0.0 ? 1.0 / xn : 0.0, 0.0);
          const double2 tw = red[a.i2];
          const double f = (rn > 0.0 && xn > 0.0) ? 1.0 / (rn * xn) : 0.0;
          st->delta_prev = st->delta;
          st->delta = make_double2(tw.x * f, tw.y * f);
          st->rho_k = rn;
          st->xi_k = xn;
        }
      }
      break;
    }
    case PH_QMR_MON: {
      monitor(a, sqrt(red[a.i0].x));
      if (is_done(st)) break;
      if (threadIdx.x == 0 && (st->rho_n == 0.0 || st->xi_n == 0.0)) { st->status = ST_BREAKDOWN; st->done = 1; }
      break;
    }
    // ------------------------------------------------------------ Li-QMR (one scalar QMR per column)
    // per-column state in slot SL_TMP5: field f of column c at [f * s + c]
    case PH_LQ_INIT: {  // i0 ||r_c||^2, i1 ||w_c||^2 (column-wise)
      if (threadIdx.x == 0) {
        double2* Q = SLP(a, SL_TMP5);
        for (int c = 0; c < s; ++c) {
          const double rho = sqrt(red[a.i0 + c].x), xi = sqrt(red[a.i1 + c].x);
          if (!isfinite(rho) || !isfinite(xi)) { st->status = ST_NAN; st->done = 1; break; }
          if (rho == 0.0 || xi == 0.0) { st->status = ST_BREAKDOWN; st->done = 1; break; }
          Q[LQ_RHO * s + c] = make_double2(rho, 0.0);
          Q[LQ_XI * s + c] = make_double2(xi, 0.0);
          Q[LQ_T * s + c] = make_double2(rho, 0.0);
          SLP(a, SL_INVRHO)[c] = make_double2(1.0 / rho, 0.0);
          SLP(a, SL_INVXI)[c] = make_double2(1.0 / xi, 0.0);
        }
        st->k = 0;
        st->have_rot1 = st->have_rot2 = 0;
      }
      break;
    }
    case PH_LQ_DELTA: {  // i0 w_c^H v_c
      if (threadIdx.x == 0) {
        double2* Q = SLP(a, SL_TMP5);
        for (int c = 0; c < s; ++c) {
          Q[LQ_DELTA * s + c] = red[a.i0 + c];
          Q[LQ_DELTAP * s + c] = make_double2(0.0, 0.0);
        }
      }
      break;
    }
    case PH_LQ_COEF1: {  // i0 w_c^H (A v_c)
      if (threadIdx.x == 0) {
        double2* Q = SLP(a, SL_TMP5);
        st->k += 1;
        for (int c = 0; c < s; ++c) {
          const double2 d = Q[LQ_DELTA * s + c];
          if (!finite2(d)) { st->status = ST_NAN; st->done = 1; break; }
          if (d.x == 0.0 && d.y == 0.0) { st->status = ST_BREAKDOWN; st->done = 1; break; }
          SLP(a, SL_ALPHA)[c] = cdiv(red[a.i0 + c], d);
          double2 be = make_double2(0.0, 0.0), ga = make_double2(0.0, 0.0);
          if (st->k >= 2) {
            const double2 q = cdiv(d, Q[LQ_DELTAP * s + c]);
            const double xi = Q[LQ_XI * s + c].x, rho = Q[LQ_RHO * s + c].x;
            be = make_double2(xi * q.x, xi * q.y);
            ga = cj(make_double2(rho * q.x, rho * q.y));
          }
          SLP(a, SL_BETA)[c] = be;
          SLP(a, SL_GAMMA)[c] = ga;
        }
      }
      break;
    }
    case PH_LQ_COEF2: {  // i0 ||vt_c||^2, i1 ||wt_c||^2, i2 wt_c^H vt_c
      if (threadIdx.x == 0) {
        double2* Q = SLP(a, SL_TMP5);
        for (int c = 0; c < s; ++c) {
          const double rn = sqrt(red[a.i0 + c].x), xn = sqrt(red[a.i1 + c].x);
          double2 u2 = make_double2(0.0, 0.0), u1 = SLP(a, SL_BETA)[c], u0 = SLP(a, SL_ALPHA)[c];
          if (st->have_rot2) {
            const double cr = Q[LQ_ROT2C * s + c].x;
            const double2 sn = Q[LQ_ROT2S * s + c];
            u2 = cm(sn, u1);
            u1 = make_double2(cr * u1.x, cr * u1.y);
          }
          if (st->have_rot1) {
            const double cr = Q[LQ_ROT1C * s + c].x;
            const double2 sn = Q[LQ_ROT1S * s + c];
            const double2 n1 = make_double2(cr * u1.x + cm(sn, u0).x, cr * u1.y + cm(sn, u0).y);
            const double2 n0 = make_double2(-cm(cj(sn), u1).x + cr * u0.x, -cm(cj(sn), u1).y + cr * u0.y);
            u1 = n1;
            u0 = n0;
          }
          double cr;
          double2 sn, ukk;
          givens(u0, make_double2(rn, 0.0), &cr, &sn, &ukk);
          if (!finite2(ukk) || !isfinite(rn) || !isfinite(xn)) { st->status = ST_NAN; st->done = 1; break; }
          if (ukk.x == 0.0 && ukk.y == 0.0) { st->status = ST_BREAKDOWN; st->done = 1; break; }
          const double2 tc = Q[LQ_T * s + c];
          const double2 tau = make_double2(cr * tc.x, cr * tc.y);
          Q[LQ_T * s + c] = neg(cm(cj(sn), tc));
          const double2 iu = cdiv(make_double2(1.0, 0.0), ukk);
          SLP(a, SL_CV)[c] = iu;
          SLP(a, SL_CD2)[c] = neg(cm(u2, iu));
          SLP(a, SL_CD1)[c] = neg(cm(u1, iu));
          SLP(a, SL_TAU)[c] = tau;
          SLP(a, SL_NTAU)[c] = neg(tau);
          Q[LQ_ROT2C * s + c] = Q[LQ_ROT1C * s + c];
          Q[LQ_ROT2S * s + c] = Q[LQ_ROT1S * s + c];
          Q[LQ_ROT1C * s + c] = make_double2(cr, 0.0);
          Q[LQ_ROT1S * s + c] = sn;
          Q[LQ_RHON * s + c] = make_double2(rn, 0.0);
          Q[LQ_XIN * s + c] = make_double2(xn, 0.0);
          SLP(a, SL_INVRHO)[c] = make_double2(rn > 0.0 ? 1.0 / rn : 0.0, 0.0);
          SLP(a, SL_INVXI)[c] = make_double2(xn > 0.0 ? 1.0 / xn : 0.0, 0.0);
          const double2 tw = red[a.i2 + c];
          const double f = (rn > 0.0 && xn > 0.0) ? 1.0 / (rn * xn) : 0.0;
          Q[LQ_DELTAP * s + c] = Q[LQ_DELTA * s + c];
          Q[LQ_DELTA * s + c] = make_double2(tw.x * f, tw.y * f);
          Q[LQ_RHO * s + c] = make_double2(rn, 0.0);
          Q[LQ_XI * s + c] = make_double2(xn, 0.0);
        }
        if (!st->done) {
          st->have_rot2 = st->have_rot1;
          st->have_rot1 = 1;
        }
      }
      break;
    }
    case PH_LQ_MON: {  // i0 ||R||_F^2
      monitor(a, sqrt(red[a.i0].x));
      if (is_done(st)) break;
      if (threadIdx.x == 0) {
        const double2* Q = SLP(a, SL_TMP5);
        for (int c = 0; c < s; ++c)
          if (Q[LQ_RHON * s + c].x == 0.0 || Q[LQ_XIN * s + c].x == 0.0) { st->status = ST_BREAKDOWN; st->done = 1; break; }
      }
      break;
    }
    // ------------------------------------------------------------ Bl-QMR
    case PH_BQ_INIT: {  // i0 W^H V; SL_RHOK = rho_0 (QR of R_0), SL_XIK = xi_1 (QR of Rh_0)
      from_red(SLP(a, SL_DELTA), red + a.i0, ss);
      copy(SLP(a, SL_T), SLP(a, SL_RHOK), ss);
      if (threadIdx.x == 0) st->k = 0;
      break;
    }
    case PH_BQ_COEF1: {  // i0 W^H Y
      double2 *T0 = SLP(a, SL_TMP0), *T1 = SLP(a, SL_TMP1), *D = SLP(a, SL_DELTA), *Dp = SLP(a, SL_DELTAP);
      if (threadIdx.x == 0) st->k += 1;
      __syncthreads();
      const int k = st->k;
      copy(T0, D, ss);
      copy(SLP(a, SL_ALPHA), red + a.i0, ss);
      if (!lu_solve(T0, SLP(a, SL_ALPHA), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      adjoint(T0, D, s);
      adjoint(SLP(a, SL_ALPHAH), red + a.i0, s);
      if (!lu_solve(T0, SLP(a, SL_ALPHAH), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      if (k >= 2) {
        matmul(SLP(a, SL_BETA), SLP(a, SL_XIK), D, s, s, s, true, false);  // xi_k^H delta_k
        copy(T0, Dp, ss);
        if (!lu_solve(T0, SLP(a, SL_BETA), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
        matmul(T1, D, SLP(a, SL_RHOK), s, s, s);                            // delta_k rho_k
        adjoint(SLP(a, SL_BETAH), T1, s);                                    // rho_k^H delta_k^H
        adjoint(T0, Dp, s);
        if (!lu_solve(T0, SLP(a, SL_BETAH), s, s, scratch, iscr)) { fail(st, ST_BREAKDOWN); break; }
      } else {
        fill(SLP(a, SL_BETA), ss, make_double2(0.0, 0.0));
        fill(SLP(a, SL_BETAH), ss, make_double2(0.0, 0.0));
      }
      break;
    }
    case PH_BQ_COEF2: {  // i0 W_new^H V_new; SL_RHON, SL_XIN from the QRs
      double2 *T0 = SLP(a, SL_TMP0), *U2 = SLP(a, SL_TMP2), *U1 = SLP(a, SL_TMP3), *U0 = SLP(a, SL_TMP4);
      double2* ST = SLP(a, SL_TMP5);
      const int k = st->k;
      fill(U2, ss, make_double2(0.0, 0.0));
      copy(U1, SLP(a, SL_BETA), ss);
      copy(U0, SLP(a, SL_ALPHA), ss);
      if (k >= 3) {
        stack2(ST, U2, U1, s);
        matmul(T0, SLP(a, SL_OM2), ST, 2 * s, 2 * s, s);
        split2(U2, U1, T0, s);
      }
      if (k >= 2) {
        stack2(ST, U1, U0, s);
        matmul(T0, SLP(a, SL_OM1), ST, 2 * s, 2 * s, s);
        split2(U1, U0, T0, s);
      }
      stack2(ST, U0, SLP(a, SL_RHON), s);
      householder_2s(SLP(a, SL_OMK), SLP(a, SL_UKK), ST, s, hv, scratch);
      const double nU = fro(SLP(a, SL_UKK), ss, scratch);
      bool bad = !isfinite(nU);
      for (int i = 0; i < s; ++i) bad = bad || cabsd(SLP(a, SL_UKK)[i * s + i]) <= 64.0 * kEps * fmax(nU, 1e-300);
      if (bad) { fail(st, ST_BREAKDOWN); break; }
      // [tau; t] = Om_k [t; 0]
      fill(T0, ss, make_double2(0.0, 0.0));
      stack2(ST, SLP(a, SL_T), T0, s);
      matmul(T0, SLP(a, SL_OMK), ST, 2 * s, 2 * s, s);
      split2(SLP(a, SL_TAU), SLP(a, SL_T), T0, s);
      scale_mat(SLP(a, SL_NTAU), SLP(a, SL_TAU), make_double2(-1.0, 0.0), ss);
      tri_inv_upper(SLP(a, SL_UKINV), SLP(a, SL_UKK), s);
      copy(SLP(a, SL_CV), SLP(a, SL_UKINV), ss);
      matmul(SLP(a, SL_CD2), U2, SLP(a, SL_UKINV), s, s, s, false, false, -1.0);
      matmul(SLP(a, SL_CD1), U1, SLP(a, SL_UKINV), s, s, s, false, false, -1.0);
      copy(SLP(a, SL_OM2), SLP(a, SL_OM1), 4 * ss);
      copy(SLP(a, SL_OM1), SLP(a, SL_OMK), 4 * ss);
      copy(SLP(a, SL_DELTAP), SLP(a, SL_DELTA), ss);
      copy(SLP(a, SL_DELTA), red + a.i0, ss);
      copy(SLP(a, SL_RHOK), SLP(a, SL_RHON), ss);
      copy(SLP(a, SL_XIK), SLP(a, SL_XIN), ss);
      break;
    }
    case PH_BQ_MON: {
      monitor(a, sqrt(red[a.i0].x));
      break;
    }
    default:
      break;
  }
}

void launch_coef(const CoefArgs& a, cudaStream_t st) {
  ProfToken tk = prof_begin(KC_COEF, st);
  coef_kernel<<<1, 256, 0, st>>>(a);
  KR_CUDA(cudaGetLastError());
  prof_end(tk, st, 0.0, 0.0);
}

}  // namespace kr
