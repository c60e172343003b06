// Plain fused step: one thread per interior cell, neighbours read straight
// from global memory.  This is the double-precision path (and a float
// variant of the same code).  Per cell and per velocity i (Secs. 2-3):
//   moments -> f^eq -> NND convection along every axis with v_ia != 0 ->
//   lambda_i Laplacian (i = 0..6) -> BGK + forward Euler, written to fout.
#include "lbm_internal.cuh"

namespace lbm {
namespace {

template <typename R>
__device__ __forceinline__ R ld(const R* __restrict__ p, long long k) {
  return __ldg(p + k);
}

template <typename R, int SCHEME>
__global__ void __launch_bounds__(256) step_plain_kernel(const R* __restrict__ fin, R* __restrict__ fout, Layout L,
                                                         Model<R> m, unsigned* __restrict__ flags) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L.nx || y >= L.ny) return;
  const long long c = L.at(x, y, z);
  const long long step[3] = {1, (long long)L.sx, L.plane};

  R f[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) f[i] = ld(fin, i * L.fs + c);

  R rho, ux, uy, uz, T;
  moments(m, f, rho, ux, uy, uz, T);
  {
    unsigned bad = 0u;
    if (!(rho > R(0))) bad |= LBM_HEALTH_RHO;
    if (!(T > R(0))) bad |= LBM_HEALTH_T;
    if (!(fabs(rho) + fabs(T) + fabs(ux) + fabs(uy) + fabs(uz) < R(1e30))) bad |= LBM_HEALTH_NONFINITE;
    if (bad) atomicOr(flags, bad);
  }
  R feq[NV];
  equilibrium(m, rho, ux, uy, uz, T, feq);

#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const R* __restrict__ p = fin + i * L.fs + c;
    const R fc = f[i];
    R conv = R(0), nb = R(0);  // nb: the six neighbours' sum (dissipation, i <= 6)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int sg = vsign(i, a);
      const long long d = step[a];
      if (sg > 0) {
        const R m2 = ld(p, -2 * d), m1 = ld(p, -d), p1 = ld(p, d);
        conv += grad_pos<SCHEME>(m2, m1, fc, p1);
        if (i <= 6) nb += p1 + m1;
      } else if (sg < 0) {
        const R m1 = ld(p, -d), p1 = ld(p, d), p2 = ld(p, 2 * d);
        conv -= grad_neg<SCHEME>(m1, fc, p1, p2);
        if (i <= 6) nb += p1 + m1;
      } else if (i <= 6) {
        const R m1 = ld(p, -d), p1 = ld(p, d);
        nb += p1 + m1;
      }
    }
    const R k = i == 0 ? R(0) : (i <= 6 ? m.k1 : m.k2);
    const R lam = i == 0 ? m.lam0 : (i <= 6 ? m.lam1 : R(0));
    // f + dt/tau (f^eq - f) - (|v| dt/dx) conv + (lambda dt/dx^2)(nb - 6 f), with the
    // relaxation and the Laplacian's centre folded into keep = 1 - dt/tau - 6 lambda dt/dx^2;
    // conv holds sum_a sign(v_ia) * grad, the velocity magnitude is in k
    const R keep = i == 0 ? m.keep0 : (i <= 6 ? m.keep1 : m.keep2);
    R o = keep * fc + m.dt_tau * feq[i];
    if (i != 0) o -= k * conv;
    if (i <= 6) o += lam * nb;
    fout[i * L.fs + c] = o;
  }
}

template <typename R>
cudaError_t launch_typed(int scheme, const R* fin, R* fout, const Layout& L, const Model<R>& m, unsigned* flags,
                         cudaStream_t st) {
  dim3 block(32, 8, 1);
  dim3 grid((L.nx + 31) / 32, (L.ny + 7) / 8, L.nz);
  switch (scheme) {
    case LBM_SCHEME_NND: step_plain_kernel<R, LBM_SCHEME_NND><<<grid, block, 0, st>>>(fin, fout, L, m, flags); break;
    case LBM_SCHEME_UPWIND2:
      step_plain_kernel<R, LBM_SCHEME_UPWIND2><<<grid, block, 0, st>>>(fin, fout, L, m, flags);
      break;
    default: step_plain_kernel<R, LBM_SCHEME_UPWIND1><<<grid, block, 0, st>>>(fin, fout, L, m, flags); break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_plain(int prec, int scheme, const void* fin, void* fout, const Layout& L,
                              const Model<double>& md, const Model<float>& mf, unsigned* flags, cudaStream_t st) {
  if (prec == LBM_FP64) return launch_typed<double>(scheme, (const double*)fin, (double*)fout, L, md, flags, st);
  return launch_typed<float>(scheme, (const float*)fin, (float*)fout, L, mf, flags, st);
}

}  // namespace lbm
