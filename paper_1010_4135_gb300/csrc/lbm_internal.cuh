// Internal declarations of the D3V15 FD-LB CUDA library (sm_103a).
//
// Device layout of one f buffer (element type R = double or float):
//   f[i][zp][yp][xp] with xp = x + OX, yp = y + 2, zp = z + 2 for interior
//   cell (x, y, z); rows of sx elements (sx a multiple of 32), planes of
//   sx*(ny+4) elements, fields fs elements apart.  Two node layers surround
//   the interior on every face (the paper's nodes 0,1 and NX,NX+1, Sec. 4(2)).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm.h"

namespace lbm {

constexpr int NV = 15;
// x offset of the first interior cell inside a padded row: OX - 2 is a
// multiple of 4, so a tile's first halo column (x0 + OX - 2, x0 a multiple of
// 32) starts on a 16-byte boundary as a TMA copy requires.
constexpr int OX = 6;

// Sign pattern of the discrete velocities (Sec. 2), index order of lbm.h.
// Magnitude: 0 for i = 0, c1 for i = 1..6, c2/sqrt(3) for i = 7..14.
__host__ __device__ constexpr int vsign(int i, int a) {
  return i == 0 ? 0
       : i <= 6 ? ((i - 1) / 2 == a ? ((i - 1) % 2 == 0 ? 1 : -1) : 0)
                : (((i - 7) >> (2 - a)) & 1 ? -1 : 1);
}

struct Layout {
  int nx, ny, nz;
  int sx;             // row pitch (elements)
  long long plane;    // sx * (ny + 4)
  long long fs;       // field stride (elements)
  __host__ __device__ long long at(int x, int y, int z) const {
    return (long long)(z + 2) * plane + (long long)(y + 2) * sx + (long long)(x + OX);
  }
  __host__ __device__ long long ncell() const { return (long long)nx * ny * nz; }
};

// Equilibrium and step constants, precomputed on the host in double.
// Per shell the paper's coefficients (Eq. "eq") are affine in T and u^2:
//   A = A0 + AT*T + AU*u^2,  B = B0 + BT*T + BU*u^2,  D constant,
// rest particle: A = AR*T, B = D = 0.
template <typename R>
struct Model {
  R c1, s, eta0sq, c1sq, c2sq, inv_b;
  R AR;
  R Aa0, AaT, AaU, Ba0, BaT, BaU, Da;  // axis shell, i = 1..6
  R Ad0, AdT, AdU, Bd0, BdT, BdU, Dd;  // diagonal shell, i = 7..14
  R dt_tau;   // dt / tau
  R k1, k2;   // c1 dt/dx, (c2/sqrt 3) dt/dx
  R lam0, lam1;  // lambda_i dt/dx^2 for i = 0 and i = 1..6 (0 when the term is off)
};

struct BcDesc {
  int kind[6];          // face 2a+hi: LBM_BC_*
  double fixed[6][5];   // (rho,u1,u2,u3,T)
};

// ---------------------------------------------------------------- physics

// Moments of 15 values (relations e1-e3): rho, u, T with
// E = eta0^2 f0 + c1^2 sum_{axis} f + c2^2 sum_{diag} f, T = (E/rho - u^2)/b.
template <typename R, typename M>
__host__ __device__ __forceinline__ void moments(const M& m, const R f[NV], R& rho, R& ux, R& uy, R& uz, R& T) {
  const R sa = ((f[1] + f[2]) + (f[3] + f[4])) + (f[5] + f[6]);
  const R dpp = f[7] + f[8], dpm = f[9] + f[10], dmp = f[11] + f[12], dmm = f[13] + f[14];
  const R sd = (dpp + dpm) + (dmp + dmm);
  rho = f[0] + sa + sd;
  const R mx = m.c1 * (f[1] - f[2]) + m.s * ((dpp + dpm) - (dmp + dmm));
  const R my = m.c1 * (f[3] - f[4]) + m.s * ((dpp + dmp) - (dpm + dmm));
  const R mz = m.c1 * (f[5] - f[6]) + m.s * (((f[7] + f[9]) + (f[11] + f[13])) - ((f[8] + f[10]) + (f[12] + f[14])));
  const R E = m.eta0sq * f[0] + m.c1sq * sa + m.c2sq * sd;
  const R ir = R(1) / rho;
  ux = mx * ir;
  uy = my * ir;
  uz = mz * ir;
  T = (E * ir - (ux * ux + uy * uy + uz * uz)) * m.inv_b;
}

// f^eq_i = rho (A_i + B_i w + D_i w^2), w = v_i . u (Eq. "eq").
template <typename R, typename M>
__host__ __device__ __forceinline__ void equilibrium(const M& m, R rho, R ux, R uy, R uz, R T, R feq[NV]) {
  const R usq = ux * ux + uy * uy + uz * uz;
  feq[0] = rho * (m.AR * T);
  const R Aa = m.Aa0 + m.AaT * T + m.AaU * usq;
  const R Ba = m.Ba0 + m.BaT * T + m.BaU * usq;
  const R u3[3] = {ux, uy, uz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R w = m.c1 * u3[a];
    const R q = Aa + m.Da * (w * w);
    const R l = Ba * w;
    feq[1 + 2 * a] = rho * (q + l);
    feq[2 + 2 * a] = rho * (q - l);
  }
  const R Ad = m.Ad0 + m.AdT * T + m.AdU * usq;
  const R Bd = m.Bd0 + m.BdT * T + m.BdU * usq;
  // k = 0..3 are (+ + +), (+ + -), (+ - +), (+ - -); k and 7-k are opposite
  const R w4[4] = {m.s * ((ux + uy) + uz), m.s * ((ux + uy) - uz), m.s * ((ux - uy) + uz), m.s * ((ux - uy) - uz)};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const R w = w4[k];
    const R q = Ad + m.Dd * (w * w);
    const R l = Bd * w;
    feq[7 + k] = rho * (q + l);
    feq[14 - k] = rho * (q - l);
  }
}

// minmod(a, b): the argument of smaller magnitude when both have the same
// sign, else 0 (the paper's 1/2 min(|X|,|Y|)(Sign X + Sign Y), Sec. 3).
template <typename R>
__device__ __forceinline__ R minmod(R a, R b) {
  return fmax(fmin(a, b), R(0)) + fmin(fmax(a, b), R(0));
}
__device__ __forceinline__ float minmod(float a, float b) {
  return fmaxf(fminf(a, b), 0.0f) + fminf(fmaxf(a, b), 0.0f);
}

// dx * d(v f)/dx / v along one axis, from the upwind-side stencil:
// v > 0 uses f at I-2..I+1 (m2, m1, c, p1); v < 0 uses I-1..I+2 (m1, c, p1, p2).
// NND: (h_{I+1/2} - h_{I-1/2}) / v with the limited fluxes of Sec. 3.
template <int SCHEME, typename R>
__device__ __forceinline__ R grad_pos(R m2, R m1, R c, R p1) {
  if (SCHEME == LBM_SCHEME_UPWIND1) return c - m1;
  if (SCHEME == LBM_SCHEME_UPWIND2) return R(0.5) * ((R(3) * c - R(4) * m1) + m2);
  const R d0 = c - m1;
  return d0 + R(0.5) * (minmod(p1 - c, d0) - minmod(d0, m1 - m2));
}
template <int SCHEME, typename R>
__device__ __forceinline__ R grad_neg(R m1, R c, R p1, R p2) {
  if (SCHEME == LBM_SCHEME_UPWIND1) return p1 - c;
  if (SCHEME == LBM_SCHEME_UPWIND2) return R(0.5) * ((R(4) * p1 - R(3) * c) - p2);
  const R d1 = p1 - c;
  return d1 - R(0.5) * (minmod(d1, p2 - p1) - minmod(c - m1, d1));
}

// ---------------------------------------------------------------- launchers
// Each returns cudaGetLastError() after enqueueing on `st`.

cudaError_t launch_fill(int prec, void* f, const Layout& L, const Model<double>& m, const BcDesc& bc, cudaStream_t st);
cudaError_t launch_init(int prec, void* f, const Layout& L, const Model<double>& m, const double* rho,
                        const double* u, const double* T, cudaStream_t st);
cudaError_t launch_moments(int prec, const void* f, const Layout& L, const Model<double>& m, double* rho, double* u,
                           double* T, cudaStream_t st);
cudaError_t launch_pack(int prec, const void* f, const Layout& L, void* dense, cudaStream_t st);
cudaError_t launch_unpack(int prec, void* f, const Layout& L, const void* dense, cudaStream_t st);
cudaError_t launch_conserved(int prec, const void* f, const Layout& L, const Model<double>& m, double* partials,
                             int max_blocks, unsigned* counter, double* result, unsigned* flags, cudaStream_t st);
cudaError_t launch_step_plain(int prec, int scheme, const void* fin, void* fout, const Layout& L,
                              const Model<double>& md, const Model<float>& mf, unsigned* flags, cudaStream_t st);
cudaError_t launch_step_tiled(int scheme, const CUtensorMap& map, const float* fin, float* fout, const Layout& L,
                              const Model<float>& m, int zc, unsigned* flags, cudaStream_t st);
// Geometry of the tiled kernel's TMA box (x, y extents) and CTA tile.
int tiled_box_x();
int tiled_box_y();
constexpr int kTileX = 32, kTileY = 8;

}  // namespace lbm
