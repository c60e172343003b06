// Boundary fill, initialisation, moments, pack/unpack and the FP64
// conservation reduction.  Initialisation and moments compute in double
// precision whatever the storage type of f; the boundary fill computes in the
// storage precision (its results are stored at that precision).
#include "lbm_internal.cuh"

namespace lbm {
namespace {

template <typename R>
__device__ __forceinline__ void load_cell(const R* __restrict__ f, long long fs, long long idx, double v[NV]) {
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = (double)f[i * fs + idx];
}

template <typename R>
__device__ __forceinline__ void store_cell(R* __restrict__ f, long long fs, long long idx, const double v[NV]) {
#pragma unroll
  for (int i = 0; i < NV; ++i) f[i * fs + idx] = (R)v[i];
}

__device__ __forceinline__ void macros_at(const Model<double>& m, const double v[NV], double out[5]) {
  double rho, ux, uy, uz, T;
  moments(m, v, rho, ux, uy, uz, T);
  out[0] = rho; out[1] = ux; out[2] = uy; out[3] = uz; out[4] = T;
}

// Error-free sum of two floats: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// Running sum of floats held as an unevaluated pair hi + lo (about 44
// significant bits).  add() keeps hi the rounded running sum and adds its
// rounding error (exact, two_sum) to lo; renorm() folds lo back into hi
// (|hi| >= |lo|, so the fast two-sum is exact) and is called every few adds,
// so lo stays of order 2^-24 |hi| and n additions lose about n * 2^-48
// relative.
struct DFloat {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
  }
  __device__ __forceinline__ void renorm() {
    const float s = hi + lo;
    lo = lo - (s - hi);
    hi = s;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// One thread per (face position): writes the two node layers outside a face.
// blockIdx.y = face (2*axis + hi); faces whose bit is clear in `mask` are
// skipped.  Sec. 4(2) boundary rules, ghost f = f^eq.  M is the arithmetic
// type (the storage type of f: ghost values are stored at that precision).
template <typename R, typename M>
__global__ void fill_kernel(R* __restrict__ f, Layout L, Model<M> m, BcDesc bc, unsigned mask) {
  const int face = blockIdx.y;
  if (!((mask >> face) & 1u)) return;
  const int axis = face >> 1, hi = face & 1;
  // cross-section coordinates (s1 fastest) and the element stride along the face normal
  const int n1 = axis == 0 ? L.ny : L.nx;
  const int n2 = axis == 2 ? L.ny : L.nz;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)n1 * n2) return;
  const int s1 = (int)(p % n1), s2 = (int)(p / n1);
  const long long base = axis == 0 ? L.at(0, s1, s2) : (axis == 1 ? L.at(s1, 0, s2) : L.at(s1, s2, 0));
  const long long step = axis == 0 ? 1LL : (axis == 1 ? (long long)L.sx : L.plane);
  const int N = axis == 0 ? L.nx : (axis == 1 ? L.ny : L.nz);
  const int kind = bc.kind[face];
  const int g1 = hi ? N : -1, g2 = hi ? N + 1 : -2;
  const long long i1 = base + g1 * step, i2 = base + g2 * step;
  if (kind == LBM_BC_PERIODIC) {
    const long long r1 = base + (((g1 % N) + N) % N) * step, r2 = base + (((g2 % N) + N) % N) * step;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const R v1 = f[i * L.fs + r1], v2 = f[i * L.fs + r2];
      f[i * L.fs + i1] = v1;
      f[i * L.fs + i2] = v2;
    }
    return;
  }
  M G1[5], G2[5];
  if (kind == LBM_BC_FIXED) {
#pragma unroll
    for (int k = 0; k < 5; ++k) G1[k] = G2[k] = (M)bc.fixed[face][k];
  } else {
    const long long m0 = base + (hi ? N - 1 : 0) * step;
    M v[NV], M0[5];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = (M)f[i * L.fs + m0];
    moments(m, v, M0[0], M0[1], M0[2], M0[3], M0[4]);
    if (kind == LBM_BC_EXTRAPOLATE) {
      const long long m1 = base + (hi ? N - 2 : 1) * step;
      M M1[5];
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] = (M)f[i * L.fs + m1];
      moments(m, v, M1[0], M1[1], M1[2], M1[3], M1[4]);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        G1[k] = M(2) * M0[k] - M1[k];
        G2[k] = M(2) * G1[k] - M0[k];
      }
    } else {  // LBM_BC_REFLECT: the normal velocity is component 1 + axis
#pragma unroll
      for (int k = 0; k < 5; ++k) G1[k] = G2[k] = M0[k];
      const M un = axis == 0 ? M0[1] : (axis == 1 ? M0[2] : M0[3]);
      if (axis == 0) { G1[1] = M(0); G2[1] = -un; }
      if (axis == 1) { G1[2] = M(0); G2[2] = -un; }
      if (axis == 2) { G1[3] = M(0); G2[3] = -un; }
    }
  }
  M e[NV];
  equilibrium(m, G1[0], G1[1], G1[2], G1[3], G1[4], e);
#pragma unroll
  for (int i = 0; i < NV; ++i) f[i * L.fs + i1] = (R)e[i];
  equilibrium(m, G2[0], G2[1], G2[2], G2[3], G2[4], e);
#pragma unroll
  for (int i = 0; i < NV; ++i) f[i * L.fs + i2] = (R)e[i];
}

__device__ __forceinline__ bool cell_of(const Layout& L, long long k, int& x, int& y, int& z) {
  if (k >= L.ncell()) return false;
  x = (int)(k % L.nx);
  const long long r = k / L.nx;
  y = (int)(r % L.ny);
  z = (int)(r / L.ny);
  return true;
}

template <typename R>
__global__ void init_kernel(R* __restrict__ f, Layout L, Model<double> m, const double* __restrict__ rho,
                            const double* __restrict__ u, const double* __restrict__ T) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!cell_of(L, k, x, y, z)) return;
  const long long n = L.ncell();
  double e[NV];
  equilibrium(m, rho[k], u[k], u[n + k], u[2 * n + k], T[k], e);
  store_cell(f, L.fs, L.at(x, y, z), e);
}

template <typename R>
__global__ void moments_kernel(const R* __restrict__ f, Layout L, Model<double> m, double* __restrict__ rho,
                               double* __restrict__ u, double* __restrict__ T) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!cell_of(L, k, x, y, z)) return;
  const long long n = L.ncell();
  double v[NV], mm[5];
  load_cell(f, L.fs, L.at(x, y, z), v);
  macros_at(m, v, mm);
  rho[k] = mm[0];
  u[k] = mm[1];
  u[n + k] = mm[2];
  u[2 * n + k] = mm[3];
  T[k] = mm[4];
}

template <typename R>
__global__ void pack_kernel(const R* __restrict__ f, Layout L, R* __restrict__ dense) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!cell_of(L, k, x, y, z)) return;
  const long long n = L.ncell(), idx = L.at(x, y, z);
#pragma unroll
  for (int i = 0; i < NV; ++i) dense[i * n + k] = f[i * L.fs + idx];
}

template <typename R>
__global__ void unpack_kernel(R* __restrict__ f, Layout L, const R* __restrict__ dense) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!cell_of(L, k, x, y, z)) return;
  const long long n = L.ncell(), idx = L.at(x, y, z);
#pragma unroll
  for (int i = 0; i < NV; ++i) f[i * L.fs + idx] = dense[i * n + k];
}

// Two x-columns of every (y, z) row and field against a dense [15][nz][ny][2]
// array: to_dense = 1 copies the interior columns next to the x face `side`
// (x = 0, 1 or nx-2, nx-1) out, to_dense = 0 writes the two layers outside it
// (x = -2, -1 or nx, nx+1).  One thread per (field, row, column).
template <typename R>
__global__ void halo_kernel(R* __restrict__ f, Layout L, int side, int to_dense, R* __restrict__ dense) {
  const long long rows = (long long)L.ny * L.nz;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= rows * 2 * NV) return;
  const int j = (int)(k & 1);
  const long long r = (k >> 1) % rows;
  const int i = (int)((k >> 1) / rows);
  const int y = (int)(r % L.ny), z = (int)(r / L.ny);
  const int x = to_dense ? (side ? L.nx - 2 + j : j) : (side ? L.nx + j : -2 + j);
  const long long at = (long long)i * L.fs + L.at(x, y, z);
  if (to_dense) dense[k] = f[at];
  else f[at] = dense[k];
}

// conservation sums: blocks of 12 warps, 4 row slots x 3 groups of 5 fields
constexpr int RED_GROUPS = 3, RED_GF = NV / RED_GROUPS, RED_ROWS = 4;
constexpr int RED_THREADS = 32 * RED_GROUPS * RED_ROWS;
static_assert(RED_GROUPS * RED_GF == NV, "field groups cover the 15 fields");

__device__ __forceinline__ bool finite_value(double v) { return fabs(v) < 1e300; }
__device__ __forceinline__ bool finite_value(float v) { return fabsf(v) < 3.0e38f; }

// Per-field accumulation of one thread's cells: double for double storage;
// for float storage an error-free double-float pair, converted to double at
// the end (GB300's FP64 rate would make a per-value conversion and double
// add the bottleneck of this memory-bound reduction).
template <typename R, int N>
struct FieldAcc;
template <int N>
struct FieldAcc<double, N> {
  double s[N];
  __device__ FieldAcc() {
#pragma unroll
    for (int i = 0; i < N; ++i) s[i] = 0.0;
  }
  __device__ __forceinline__ void add(int i, double v) { s[i] += v; }
  __device__ __forceinline__ void renorm() {}
  __device__ __forceinline__ double value(int i) const { return s[i]; }
};
template <int N>
struct FieldAcc<float, N> {
  DFloat s[N];
  __device__ __forceinline__ void add(int i, float v) { s[i].add(v); }
  __device__ __forceinline__ void renorm() {
#pragma unroll
    for (int i = 0; i < N; ++i) s[i].renorm();
  }
  __device__ __forceinline__ double value(int i) const { return s[i].value(); }
};

// 16-byte vector loads of float / double rows (read once: streaming hint).
__device__ __forceinline__ void load16(const float* p, float v[4]) {
  const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load16(const double* p, double v[2]) {
  const double2 q = __ldcs(reinterpret_cast<const double2*>(p));
  v[0] = q.x; v[1] = q.y;
}

// Deterministic FP64 global sums of (rho, rho u, E) over interior cells.  The
// moments are linear in f, so the kernel sums each field f_i over the cells
// and combines the 15 field totals at the end: mass = sum_i F_i, momentum =
// sum_i v_i F_i, energy = sum_i (v_i^2 + eta_i^2) F_i.  Each warp takes whole
// x rows (rows b * RED_ROWS + slot, stepping by gridDim.x * RED_ROWS) and one
// group of five fields, three warps per row slot; a lane reads 16 bytes of
// each of its five fields per x step (a warp: 512 contiguous bytes per
// field), all five loads issued before the first add.  Few registers per
// thread let many warps, and so many bytes, be in flight per SM.  Values
// past the row end are masked to zero.  Warps reduce by a fixed shuffle
// tree, blocks by warp order, and the last block to finish sums the
// per-block totals with 256 of its threads in a fixed split (16 strided
// partial sums per field, then in order).  The order never depends on
// timing, so the result is bitwise reproducible for a given grid.
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) conserved_kernel(const R* __restrict__ f, Layout L, Model<double> m,
                                                                double* __restrict__ partials,
                                                                unsigned* __restrict__ counter,
                                                                double* __restrict__ result,
                                                                unsigned* __restrict__ flags) {
  constexpr int WARPS = RED_THREADS / 32;
  __shared__ double wsum[WARPS][16];
  __shared__ double part[16][16];
  __shared__ bool last;
  FieldAcc<R, RED_GF> acc;
  bool bad = false;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = warp % RED_GROUPS, slot = warp / RED_GROUPS;
  const int nrows = L.ny * L.nz;
  const int nr = gridDim.x * RED_ROWS;
  constexpr int VW = 16 / (int)sizeof(R);  // elements per 16-byte load
  const R* fg = f + (long long)grp * RED_GF * L.fs;
  for (int r = blockIdx.x * RED_ROWS + slot; r < nrows; r += nr) {
    // interior rows start at x = OX (a multiple of 8 elements): 16-byte aligned
    const R* row = fg + L.at(0, r % L.ny, r / L.ny);
    for (int x0 = lane * VW; x0 < L.nx; x0 += 32 * VW) {
      // the last vector may reach up to VW - 1 elements past the row end,
      // into the row's halo and padding (inside the buffer); masked below
      R v[RED_GF][VW];
#pragma unroll
      for (int i = 0; i < RED_GF; ++i) load16(row + i * L.fs + x0, v[i]);
#pragma unroll
      for (int i = 0; i < RED_GF; ++i) {
#pragma unroll
        for (int k = 0; k < VW; ++k) {
          const R e = x0 + k < L.nx ? v[i][k] : R(0);
          bad |= !finite_value(e);
          acc.add(i, e);
        }
      }
      acc.renorm();
    }
  }
  if (bad) atomicOr(flags, (unsigned)LBM_HEALTH_NONFINITE);
#pragma unroll
  for (int i = 0; i < RED_GF; ++i) {
    double v = acc.value(i);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) wsum[warp][grp * RED_GF + i] = v;
  }
  // the other groups' fields of this warp are zero (adding them is exact)
  if (lane < NV && (lane < grp * RED_GF || lane >= (grp + 1) * RED_GF)) wsum[warp][lane] = 0.0;
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) t += wsum[w][threadIdx.x];
    partials[blockIdx.x * 16 + threadIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 256) {
    // field i, strided part j of 16; the partials are read through L2 (the
    // other blocks' writes are ordered before their counter increments),
    // eight loads in flight per step of the fixed-order sum
    const int i = threadIdx.x & 15, j = threadIdx.x >> 4;
    double t = 0.0;
    if (i < NV) {
      unsigned b = j;
      for (; b + 7 * 16 < gridDim.x; b += 8 * 16) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __ldcg(partials + (b + q * 16) * 16 + i);
#pragma unroll
        for (int q = 0; q < 8; ++q) t += v[q];
      }
      for (; b < gridDim.x; b += 16) t += __ldcg(partials + b * 16 + i);
    }
    part[j][i] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double F[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      F[i] = 0.0;
      for (int j = 0; j < 16; ++j) F[i] += part[j][i];
    }
    const double sa = ((F[1] + F[2]) + (F[3] + F[4])) + (F[5] + F[6]);
    const double sd = ((F[7] + F[8]) + (F[9] + F[10])) + ((F[11] + F[12]) + (F[13] + F[14]));
    result[0] = F[0] + sa + sd;
    result[1] = m.c1 * (F[1] - F[2]) + m.s * (((F[7] + F[8]) + (F[9] + F[10])) - ((F[11] + F[12]) + (F[13] + F[14])));
    result[2] = m.c1 * (F[3] - F[4]) + m.s * (((F[7] + F[8]) + (F[11] + F[12])) - ((F[9] + F[10]) + (F[13] + F[14])));
    result[3] = m.c1 * (F[5] - F[6]) + m.s * (((F[7] + F[9]) + (F[11] + F[13])) - ((F[8] + F[10]) + (F[12] + F[14])));
    result[4] = m.eta0sq * F[0] + m.c1sq * sa + m.c2sq * sd;
    *counter = 0u;
  }
}

inline int blocks_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_fill(int prec, void* f, const Layout& L, const Model<double>& md, const Model<float>& mf,
                        const BcDesc& bc, unsigned mask, cudaStream_t st) {
  if (!mask) return cudaSuccess;
  long long cmax = 1;
  const long long cnt[3] = {(long long)L.ny * L.nz, (long long)L.nx * L.nz, (long long)L.nx * L.ny};
  for (int a = 0; a < 3; ++a)
    if (((mask >> (2 * a)) & 3u) && cnt[a] > cmax) cmax = cnt[a];
  dim3 grid((unsigned)((cmax + 127) / 128), 6);
  if (prec == LBM_FP64) fill_kernel<double, double><<<grid, 128, 0, st>>>((double*)f, L, md, bc, mask);
  else fill_kernel<float, float><<<grid, 128, 0, st>>>((float*)f, L, mf, bc, mask);
  return cudaGetLastError();
}

cudaError_t launch_init(int prec, void* f, const Layout& L, const Model<double>& m, const double* rho, const double* u,
                        const double* T, cudaStream_t st) {
  const int b = blocks_for(L.ncell(), 256);
  if (prec == LBM_FP64) init_kernel<double><<<b, 256, 0, st>>>((double*)f, L, m, rho, u, T);
  else init_kernel<float><<<b, 256, 0, st>>>((float*)f, L, m, rho, u, T);
  return cudaGetLastError();
}

cudaError_t launch_moments(int prec, const void* f, const Layout& L, const Model<double>& m, double* rho, double* u,
                           double* T, cudaStream_t st) {
  const int b = blocks_for(L.ncell(), 256);
  if (prec == LBM_FP64) moments_kernel<double><<<b, 256, 0, st>>>((const double*)f, L, m, rho, u, T);
  else moments_kernel<float><<<b, 256, 0, st>>>((const float*)f, L, m, rho, u, T);
  return cudaGetLastError();
}

cudaError_t launch_pack(int prec, const void* f, const Layout& L, void* dense, cudaStream_t st) {
  const int b = blocks_for(L.ncell(), 256);
  if (prec == LBM_FP64) pack_kernel<double><<<b, 256, 0, st>>>((const double*)f, L, (double*)dense);
  else pack_kernel<float><<<b, 256, 0, st>>>((const float*)f, L, (float*)dense);
  return cudaGetLastError();
}

cudaError_t launch_unpack(int prec, void* f, const Layout& L, const void* dense, cudaStream_t st) {
  const int b = blocks_for(L.ncell(), 256);
  if (prec == LBM_FP64) unpack_kernel<double><<<b, 256, 0, st>>>((double*)f, L, (const double*)dense);
  else unpack_kernel<float><<<b, 256, 0, st>>>((float*)f, L, (const float*)dense);
  return cudaGetLastError();
}

cudaError_t launch_halo(int prec, void* f, const Layout& L, int side, int to_dense, void* dense, cudaStream_t st) {
  const int b = blocks_for((long long)L.ny * L.nz * 2 * NV, 256);
  if (prec == LBM_FP64) halo_kernel<double><<<b, 256, 0, st>>>((double*)f, L, side, to_dense, (double*)dense);
  else halo_kernel<float><<<b, 256, 0, st>>>((float*)f, L, side, to_dense, (float*)dense);
  return cudaGetLastError();
}

cudaError_t launch_conserved(int prec, const void* f, const Layout& L, const Model<double>& m, double* partials,
                             int max_blocks, unsigned* counter, double* result, unsigned* flags, cudaStream_t st) {
  // about eight rows per row slot, at most max_blocks blocks
  int b = blocks_for((long long)L.ny * L.nz, 8 * RED_ROWS);
  if (b > max_blocks) b = max_blocks;
  if (b < 1) b = 1;
  if (prec == LBM_FP64)
    conserved_kernel<double><<<b, RED_THREADS, 0, st>>>((const double*)f, L, m, partials, counter, result, flags);
  else
    conserved_kernel<float><<<b, RED_THREADS, 0, st>>>((const float*)f, L, m, partials, counter, result, flags);
  return cudaGetLastError();
}

}  // namespace lbm
