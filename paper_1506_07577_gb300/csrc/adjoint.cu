// Adjoint element map of the implicit step (FP64, St. Venant-Kirchhoff).
//
// One thread per tet.  Inputs: the state u (F = I + Du Dm^-1), the adjoint
// solution lam and w = v' (the step's new velocity).  Per tet, with
// L = Dlam Dm^-1 and W = Dw Dm^-1:
//   K lam         corners V dP(F; L) b_a                       -> acc_kl
//   d/dx[lam^T K(x) w]  corners V Q b_a, Q = d/dF [dP(F; W) : L] -> acc_xq
//     Q = 2 mu F sym(W^T L) + lam_ tr(W^T L) F + L C + 2 mu W sym(F^T L)
//         + lam_ tr(F^T L) W,   C = 2 mu sym(F^T W) + lam_ tr(F^T W) I
//   dL/dmu  += dt d/dmu[lam^T f] - dt^2 d/dmu[lam^T K w]
//            = -dt V (2 F E) : L - dt^2 V (W 2E + F 2 sym(F^T W)) : L
//   dL/dlam_ += -dt V tr(E) (F : L) - dt^2 V (tr(E) (W : L) + tr(F^T W) (F : L))
// (b_a = row a-1 of Dm^-1 for corners 1..3, corner 0 the negative sum; the
// stiffness-vector part reuses the K w element math, so the Hessian-vector
// product of the adjoint is the forward K w.)  Per-tet gradients go to the
// caller's tet order through the internal -> caller permutation.
#include "ebb_internal.h"
#include "tet_math.cuh"

namespace ebb {
namespace {

constexpr int kAdjThreads = 128;

__device__ __forceinline__ void sym3(const double* A, double* S) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) S[i * 3 + j] = 0.5 * (A[i * 3 + j] + A[j * 3 + i]);
}

__device__ __forceinline__ double ddot9(const double* A, const double* B) {
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) s += A[i] * B[i];
  return s;
}

__global__ void __launch_bounds__(kAdjThreads)
adjoint_stvk_kernel(int nt, int nv, const int4* __restrict__ keys, const int* __restrict__ perm,
                    TetStreams<double> s, double mu0, double lam0, const double* __restrict__ u,
                    const double* __restrict__ lv, const double* __restrict__ w, double* acc_kl, double* acc_xq,
                    double* gmu, double* glam, double dt) {
  const int t = blockIdx.x * kAdjThreads + threadIdx.x;
  if (t >= nt) return;
  const int4 k4 = keys[t];
  const int kk[4] = {k4.x, k4.y, k4.z, k4.w};
  double B[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i] = s.B[(size_t)i * nt + t];
  const double V = s.V[t];
  const double mu = s.mu ? s.mu[t] : mu0;
  const double lam = s.lam ? s.lam[t] : lam0;
  double Du[9], Dl[9], Dw[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double u0 = u[(size_t)c * nv + kk[0]], l0 = lv[(size_t)c * nv + kk[0]], w0 = w[(size_t)c * nv + kk[0]];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Du[c * 3 + j] = u[(size_t)c * nv + kk[j + 1]] - u0;
      Dl[c * 3 + j] = lv[(size_t)c * nv + kk[j + 1]] - l0;
      Dw[c * 3 + j] = w[(size_t)c * nv + kk[j + 1]] - w0;
    }
  }
  double G[9], L[9], W[9];
  mm(Du, B, G);
  mm(Dl, B, L);
  mm(Dw, B, W);
  StvkState<double> sv;
  stvk_state(G, mu, lam, sv);
  double F[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) F[i] = G[i] + ((i % 4) == 0 ? 1.0 : 0.0);
  // K lam: dP(F; L)
  double dPl[9];
  stvk_dP(sv, mu, lam, L, dPl);
  // Q = d/dF [dP(F; W) : L]
  double FtW[9], WtL[9], FtL[9], sWtL[9], sFtL[9], C[9];
  mtm(F, W, FtW);
  mtm(W, L, WtL);
  mtm(F, L, FtL);
  sym3(WtL, sWtL);
  sym3(FtL, sFtL);
  sym3(FtW, C);
  const double trFtW = FtW[0] + FtW[4] + FtW[8];
  const double trWtL = WtL[0] + WtL[4] + WtL[8];
  const double trFtL = FtL[0] + FtL[4] + FtL[8];
#pragma unroll
  for (int i = 0; i < 9; ++i) C[i] *= 2.0 * mu;
  C[0] += lam * trFtW;
  C[4] += lam * trFtW;
  C[8] += lam * trFtW;
  double Q[9], T1[9], T2[9], T3[9];
  mm(F, sWtL, T1);
  mm(L, C, T2);
  mm(W, sFtL, T3);
#pragma unroll
  for (int i = 0; i < 9; ++i)
    Q[i] = 2.0 * mu * T1[i] + lam * trWtL * F[i] + T2[i] + 2.0 * mu * T3[i] + lam * trFtL * W[i];
  // corners
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double s_kl = 0.0, s_xq = 0.0;
#pragma unroll
    for (int a = 1; a <= 3; ++a) {
      const double* b = B + (a - 1) * 3;
      const double kl = V * (dPl[c * 3] * b[0] + dPl[c * 3 + 1] * b[1] + dPl[c * 3 + 2] * b[2]);
      const double xq = V * (Q[c * 3] * b[0] + Q[c * 3 + 1] * b[1] + Q[c * 3 + 2] * b[2]);
      atomicAdd(acc_kl + (size_t)c * nv + kk[a], kl);
      atomicAdd(acc_xq + (size_t)c * nv + kk[a], xq);
      s_kl -= kl;
      s_xq -= xq;
    }
    atomicAdd(acc_kl + (size_t)c * nv + kk[0], s_kl);
    atomicAdd(acc_xq + (size_t)c * nv + kk[0], s_xq);
  }
  if (gmu != nullptr || glam != nullptr) {
    // E = (G + G^T + G^T G)/2
    double GtG[9], E[9];
    mtm(G, G, GtG);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) E[i * 3 + j] = 0.5 * (G[i * 3 + j] + G[j * 3 + i] + GtG[i * 3 + j]);
    const double trE = E[0] + E[4] + E[8];
    double FE[9], WE[9], FdE[9], dE[9];
    mm(F, E, FE);
    mm(W, E, WE);
    sym3(FtW, dE);
    mm(F, dE, FdE);
    const double FL = ddot9(F, L);
    const double f_mu = -V * 2.0 * ddot9(FE, L);
    const double f_lam = -V * trE * FL;
    const double k_mu = V * 2.0 * (ddot9(WE, L) + ddot9(FdE, L));
    const double k_lam = V * (trE * ddot9(W, L) + trFtW * FL);
    const int o = perm[t];
    if (gmu) gmu[o] += dt * f_mu - dt * dt * k_mu;
    if (glam) glam[o] += dt * f_lam - dt * dt * k_lam;
  }
}

}  // namespace

cudaError_t launch_adjoint_map(ebb_rel_s* rel, double mu0, double lam0, const double* u, const double* lv,
                               const double* w, double* acc_kl, double* acc_xq, double* gmu, double* glam, double dt,
                               cudaStream_t st) {
  const int nt = (int)rel->size;
  if (nt == 0) return cudaSuccess;
  adjoint_stvk_kernel<<<(nt + kAdjThreads - 1) / kAdjThreads, kAdjThreads, 0, st>>>(
      nt, (int)rel->verts->size, rel->keys, rel->tet_perm, rel->s64, mu0, lam0, u, lv, w, acc_kl, acc_xq, gmu, glam,
      dt);
  return cudaGetLastError();
}

}  // namespace ebb
