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
// x offset of the first interior cell inside a padded row.  OX is a multiple
// of 8 cells, so with row pitches that are multiples of 32 cells every tile
// row (x0 a multiple of 32) starts on a 32-byte DRAM sector: the step
// kernels' stores write whole sectors (no read-modify-write of partly
// written sectors; measured 17% faster on 256^3 than OX = 6).  The TMA boxes
// start TMA_LEFT = 4 cells left of the tile (x0 + OX - 4, 16-byte aligned as
// a TMA copy requires) and are 8 cells wider than the tile.
constexpr int OX = 8;
constexpr int TMA_LEFT = 4;
static_assert(OX % 8 == 0 && (OX - TMA_LEFT) % 4 == 0 && TMA_LEFT >= 2, "row alignment");

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
  // coefficient of f_i in the update once relaxation and the centre of the
  // Laplacian are folded in: 1 - dt/tau - 6 lambda_i dt/dx^2 (rest, axis, diagonal)
  R keep0, keep1, keep2;
};

// FP64 temperature recovery of the FP32 pair kernel.  T = (E/rho - u^2)/b
// with E = eta0^2 f_0 + c1^2 sum_axis f + c2^2 sum_diag f: when c1^2 >> T the
// equilibrium's axis and diagonal populations are large and of opposite sign,
// and E is a small difference of large terms (Sec. 2's A_i of the two shells).
// At f ~ f^eq the terms sum in magnitude to about rho (6 c1^2 |A_a| +
// 8 c2^2 |A_d| + (b-3) T) + rho u^2, so the relative rounding error of an FP32
// T is about eps_32 kappa with
//   kappa = 1 + (6 c1^2 |A_a| + 8 c2^2 |A_d| + u^2) / (b T).
// Cells with kappa > kappa_max (or T <= 0 in FP32) recompute rho, u and T from
// their 15 values in FP64.
struct RecoverDesc {
  double c1, s, eta0sq, c1sq, c2sq, inv_b;  // moment constants in FP64
  float axis_w, diag_w;                     // 6 c1^2, 8 c2^2
  float thresh_b;                           // (kappa_max - 1) b
  int on;                                   // 0: FP32 recovery everywhere
};

struct BcDesc {
  int kind[6];          // face 2a+hi: LBM_BC_*
  double fixed[6][5];   // (rho,u1,u2,u3,T)
};

// Boundary layers a step kernel writes itself for the state it produces
// ("write-through"), so that no fill kernel runs before the next step:
// periodic images along each flagged axis, and the extrapolated / reflected
// layers of the x faces (kind LBM_BC_EXTRAPOLATE or LBM_BC_REFLECT, 0 = not
// handled in the kernel).
struct WtDesc {
  int per[3];
  int xlo, xhi;
};

// ---------------------------------------------------------------- physics

// Explicitly rounded arithmetic.  Every product, sum and fused multiply-add
// below is spelled out, so the compiler contracts nothing on its own and the
// same expression rounds identically in every kernel that inlines it (the
// fill kernel, the step kernels, the write-through of the boundary layers,
// and the batched step).  The order matches the packed-pair step kernel.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Moments of 15 values (relations e1-e3): rho, u, T with
// E = eta0^2 f0 + c1^2 sum_{axis} f + c2^2 sum_{diag} f, T = (E/rho - u^2)/b.
template <typename R, typename M>
__device__ __forceinline__ void moments(const M& m, const R f[NV], R& rho, R& ux, R& uy, R& uz, R& T) {
  const R sa = radd(radd(radd(f[1], f[2]), radd(f[3], f[4])), radd(f[5], f[6]));
  const R dpp = radd(f[7], f[8]), dpm = radd(f[9], f[10]), dmp = radd(f[11], f[12]), dmm = radd(f[13], f[14]);
  const R sd = radd(radd(dpp, dpm), radd(dmp, dmm));
  rho = radd(radd(f[0], sa), sd);
  const R mx = rfma(R(m.c1), rsub(f[1], f[2]), rmul(R(m.s), rsub(radd(dpp, dpm), radd(dmp, dmm))));
  const R my = rfma(R(m.c1), rsub(f[3], f[4]), rmul(R(m.s), rsub(radd(dpp, dmp), radd(dpm, dmm))));
  const R mz = rfma(R(m.c1), rsub(f[5], f[6]),
                    rmul(R(m.s), rsub(radd(radd(f[7], f[9]), radd(f[11], f[13])),
                                      radd(radd(f[8], f[10]), radd(f[12], f[14])))));
  const R E = rfma(R(m.eta0sq), f[0], rfma(R(m.c1sq), sa, rmul(R(m.c2sq), sd)));
  const R ir = R(1) / rho;
  ux = rmul(mx, ir);
  uy = rmul(my, ir);
  uz = rmul(mz, ir);
  const R usq = rfma(ux, ux, rfma(uy, uy, rmul(uz, uz)));
  T = rmul(rsub(rmul(E, ir), usq), R(m.inv_b));
}

// f^eq_i = rho (A_i + B_i w + D_i w^2), w = v_i . u (Eq. "eq").
template <typename R, typename M>
__device__ __forceinline__ void equilibrium(const M& m, R rho, R ux, R uy, R uz, R T, R feq[NV]) {
  const R usq = rfma(ux, ux, rfma(uy, uy, rmul(uz, uz)));
  feq[0] = rmul(rho, rmul(R(m.AR), T));
  const R Aa = rfma(R(m.AaT), T, rfma(R(m.AaU), usq, R(m.Aa0)));
  const R Ba = rfma(R(m.BaT), T, rfma(R(m.BaU), usq, R(m.Ba0)));
  const R u3[3] = {ux, uy, uz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R w = rmul(R(m.c1), u3[a]);
    const R q = rfma(R(m.Da), rmul(w, w), Aa);
    const R l = rmul(Ba, w);
    feq[1 + 2 * a] = rmul(rho, radd(q, l));
    feq[2 + 2 * a] = rmul(rho, rsub(q, l));
  }
  const R Ad = rfma(R(m.AdT), T, rfma(R(m.AdU), usq, R(m.Ad0)));
  const R Bd = rfma(R(m.BdT), T, rfma(R(m.BdU), usq, R(m.Bd0)));
  // k = 0..3 are (+ + +), (+ + -), (+ - +), (+ - -); k and 7-k are opposite
  const R sxy = radd(ux, uy), dxy = rsub(ux, uy);
  const R w4[4] = {rmul(R(m.s), radd(sxy, uz)), rmul(R(m.s), rsub(sxy, uz)), rmul(R(m.s), radd(dxy, uz)),
                   rmul(R(m.s), rsub(dxy, uz))};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const R w = w4[k];
    const R q = rfma(R(m.Dd), rmul(w, w), Ad);
    const R l = rmul(Bd, w);
    feq[7 + k] = rmul(rho, radd(q, l));
    feq[14 - k] = rmul(rho, rsub(q, l));
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

// minmod(x, d) as x clamped to [min(d, 0), max(d, 0)] (exact, like the
// two-sided form); the two minmods of one cell share d, so its bounds are
// formed once.
template <typename R>
__device__ __forceinline__ R clamp_mm(R x, R lo, R hi) {
  return fmin(fmax(x, lo), hi);
}

// minmod(x, d) of two doubles from their bit patterns, on the integer pipes:
// 0 when the signs differ, else the operand of smaller magnitude (magnitudes
// of IEEE doubles order like their bit patterns without the sign, compared
// here as (high word, low word)).  The same value as the clamp form for
// finite operands (a zero result may differ in sign).  GB300 executes FP64 at
// a small fraction of its FP32 rate and a double min or max is an FP64
// comparison, so the FP64 step kernel, bound by its FP64 pipe, takes its
// minmods here.  Written on 32-bit halves: the same selection on 64-bit
// integers cost the FP64 pipe 3 more instructions per gradient.
__device__ __forceinline__ double minmod_bits(double x, double d) {
  const int hx = __double2hiint(x), hd = __double2hiint(d);
  const unsigned lx = (unsigned)__double2loint(x), ld = (unsigned)__double2loint(d);
  const int mx = hx & 0x7fffffff, md = hd & 0x7fffffff;
  const bool take_x = mx < md || (mx == md && lx <= ld);
  const bool opposite = (hx ^ hd) < 0;
  const int rh = opposite ? 0 : (take_x ? hx : hd);
  const unsigned rl = opposite ? 0u : (take_x ? lx : ld);
  return __hiloint2double(rh, (int)rl);
}

// dx * d(v f)/dx / v along one axis, from the upwind-side stencil:
// v > 0 uses f at I-2..I+1 (m2, m1, c, p1); v < 0 uses I-1..I+2 (m1, c, p1, p2).
// NND: (h_{I+1/2} - h_{I-1/2}) / v with the limited fluxes of Sec. 3; both
// minmods of the cell take the middle difference as their clamp.
template <int SCHEME, typename R>
__device__ __forceinline__ R grad_pos(R m2, R m1, R c, R p1) {
  if (SCHEME == LBM_SCHEME_UPWIND1) return c - m1;
  if (SCHEME == LBM_SCHEME_UPWIND2) return R(0.5) * ((R(3) * c - R(4) * m1) + m2);
  const R d0 = c - m1;
  if constexpr (sizeof(R) == 8) return d0 + R(0.5) * (minmod_bits(p1 - c, d0) - minmod_bits(m1 - m2, d0));
  const R lo = fmin(d0, R(0)), hi = fmax(d0, R(0));
  return d0 + R(0.5) * (clamp_mm(p1 - c, lo, hi) - clamp_mm(m1 - m2, lo, hi));
}
template <int SCHEME, typename R>
__device__ __forceinline__ R grad_neg(R m1, R c, R p1, R p2) {
  if (SCHEME == LBM_SCHEME_UPWIND1) return p1 - c;
  if (SCHEME == LBM_SCHEME_UPWIND2) return R(0.5) * ((R(4) * p1 - R(3) * c) - p2);
  const R d1 = p1 - c;
  if constexpr (sizeof(R) == 8) return d1 - R(0.5) * (minmod_bits(p2 - p1, d1) - minmod_bits(c - m1, d1));
  const R lo = fmin(d1, R(0)), hi = fmax(d1, R(0));
  return d1 - R(0.5) * (clamp_mm(p2 - p1, lo, hi) - clamp_mm(c - m1, lo, hi));
}

// ---------------------------------------------------------------- launchers
// Each returns cudaGetLastError() after enqueueing on `st`.

// Boundary layers of the faces whose bit (2*axis + hi) is set in mask.
cudaError_t launch_fill(int prec, void* f, const Layout& L, const Model<double>& md, const Model<float>& mf,
                        const BcDesc& bc, unsigned mask, cudaStream_t st);
cudaError_t launch_init(int prec, void* f, const Layout& L, const Model<double>& m, const double* rho,
                        const double* u, const double* T, cudaStream_t st);
cudaError_t launch_moments(int prec, const void* f, const Layout& L, const Model<double>& m, double* rho, double* u,
                           double* T, cudaStream_t st);
cudaError_t launch_pack(int prec, const void* f, const Layout& L, void* dense, cudaStream_t st);
cudaError_t launch_unpack(int prec, void* f, const Layout& L, const void* dense, cudaStream_t st);
// The two x-columns next to (to_dense = 1) or outside (to_dense = 0) the x
// face `side` (0 lo, 1 hi) against dense [15][nz][ny][2] (x order).
cudaError_t launch_halo(int prec, void* f, const Layout& L, int side, int to_dense, void* dense, cudaStream_t st);
cudaError_t launch_conserved(int prec, const void* f, const Layout& L, const Model<double>& m, double* partials,
                             int max_blocks, unsigned* counter, double* result, unsigned* flags, cudaStream_t st);
cudaError_t launch_step_plain(int prec, int scheme, const void* fin, void* fout, const Layout& L,
                              const Model<double>& md, const Model<float>& mf, unsigned* flags, cudaStream_t st);
cudaError_t launch_step_tiled(int scheme, const CUtensorMap& map, const float* fin, float* fout, const Layout& L,
                              const Model<float>& m, int zc, unsigned* flags, cudaStream_t st);
// Pair kernel (two cells per thread) on `cols` x 8 tiles: cols = 64 (box
// 72 x 12, one CTA per SM) or 32 (the tiled kernel's tiles and box 40 x 12,
// two CTAs per SM).  The map's box must be pair_shape(cols).bx x .by.
struct PairShape {
  int tx, ty, bx, by, threads, ctas_per_sm;
};
PairShape pair_shape(int cols);

// How the pair kernels split the z range of a tile column into chunks (one
// chunk = one unit of work, a z-march of one CTA).  With zt = 0 all chunks
// have zc planes.  With zt > 0 the first nbig = floor((nz - zt) / zc) chunks
// have zc planes and the remaining planes are split into chunks of zt: the
// short chunks come last in launch order, so the last units of a launch are
// short and the SMs finish together.
struct ZSched {
  int zc, zt, nbig, nch;  // long and short chunk length, long chunks, all chunks
  __host__ __device__ int z0(int c) const { return c < nbig ? c * zc : nbig * zc + (c - nbig) * zt; }
  __host__ __device__ int len(int c, int nz) const {
    const int l = c < nbig ? zc : zt;
    return l < nz - z0(c) ? l : nz - z0(c);
  }
};
// nz >= 1, zc >= 1; zt = 0, zt >= zc or zt >= nz: every chunk zc planes long
inline ZSched make_zsched(int nz, int zc, int zt) {
  ZSched z;
  z.zc = zc;
  if (zt <= 0 || zt >= zc || zt >= nz) {
    z.zt = zc;
    z.nch = z.nbig = (nz + zc - 1) / zc;
  } else {
    z.zt = zt;
    z.nbig = (nz - zt) / zc;
    z.nch = z.nbig + (nz - z.nbig * zc + zt - 1) / zt;
  }
  return z;
}

cudaError_t launch_step_pair(int cols, int scheme, const CUtensorMap& map, const float* fin, float* fout,
                             const Layout& L, const Model<float>& m, const WtDesc& wt, const RecoverDesc& rd,
                             const ZSched& zs, unsigned* flags, unsigned wait_limit, cudaStream_t st);

// Descriptor table of a batched step (passed by value as the kernel
// parameter): one entry per grid, units [first_unit, first_unit +
// tiles_x * tiles_y * zs.nch) in z-chunk-major order.
constexpr int kMaxBatch = 48;
struct BatchItem {
  const float* fin;
  float* fout;
  unsigned* flags;
  Layout L;
  Model<float> m;
  WtDesc wt;
  RecoverDesc rd;
  ZSched zs;
  int tiles_x, tiles_y;
  long long first_unit;
};
struct BatchTable {
  CUtensorMap map[kMaxBatch];
  BatchItem item[kMaxBatch];
  int n;
  unsigned wait_limit;
  long long total_units;
  unsigned long long* queue;  // next unit to take (0 at launch; reset by the last CTA)
  unsigned* done;             // CTAs finished (0 at launch; reset by the last CTA)
};
// Batched step over the descriptor table (`cols` x 8 tiles, maps of that box).
cudaError_t launch_step_pair_batch(int cols, int scheme, const BatchTable& tab, int grid, cudaStream_t st);
// Field-split kernel on 32 x 8 tiles (two warp groups of 128 threads per
// tile, two CTAs per SM; the 40 x 12 map of the pair kernel), single grid and
// batched; results bitwise equal to the pair kernel's.
cudaError_t launch_step_split(int scheme, const CUtensorMap& map, const float* fin, float* fout, const Layout& L,
                              const Model<float>& m, const WtDesc& wt, const RecoverDesc& rd, const ZSched& zs,
                              unsigned* flags, unsigned wait_limit, cudaStream_t st);
cudaError_t launch_step_split_batch(int scheme, const BatchTable& tab, int grid, cudaStream_t st);
// y = 1/x as the FP32 step kernels form the inverse density (device arrays).
cudaError_t launch_reciprocal_fp32(const float* x, float* y, long long n, cudaStream_t st);
// Von Neumann service: out[p] = max |omega| of G(k) (Sec. 3) over the states
// (rho, u1, u2, u3, T), directions and nk wave numbers, for each parameter
// set p = (c1, c2, eta0, gamma, dt, tau, dx); device pointers; out zeroed here.
cudaError_t launch_vn_max_growth(const double* states, int nstates, const double* params, int nparams,
                                 const double* dirs, int ndirs, int nk, int dissipation, double* out,
                                 cudaStream_t st);
// Shared-memory attributes of the tiled kernels; set once per device before
// their first launch (not allowed inside a stream capture).
cudaError_t prepare_tiled_kernels();
cudaError_t prepare_pair_kernels();
cudaError_t prepare_split_kernels();
// Geometry of the tiled kernel's TMA box (x, y extents) and CTA tile.
int tiled_box_x();
int tiled_box_y();
constexpr int kTileX = 32, kTileY = 8;

}  // namespace lbm
