// Boundary fill, initialisation, moments, pack/unpack and the FP64
// conservation reduction.  All of these work in double precision whatever
// the storage type of f.
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

// One thread per (face position): writes the two node layers outside a face.
// blockIdx.y = face (2*axis + hi).  Sec. 4(2) boundary rules, ghost f = f^eq.
template <typename R>
__global__ void fill_kernel(R* __restrict__ f, Layout L, Model<double> m, BcDesc bc) {
  const int face = blockIdx.y;
  const int axis = face >> 1, hi = face & 1;
  const int n[3] = {L.nx, L.ny, L.nz};
  const int a1 = axis == 0 ? 1 : 0;
  const int a2 = axis == 2 ? 1 : 2;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long count = (long long)n[a1] * n[a2];
  if (p >= count) return;
  int q[3];
  q[a1] = (int)(p % n[a1]);
  q[a2] = (int)(p / n[a1]);
  const int N = n[axis];
  const int kind = bc.kind[face];
  const int g1 = hi ? N : -1, g2 = hi ? N + 1 : -2;
  auto index = [&](int k) {
    int c[3] = {q[0], q[1], q[2]};
    c[axis] = k;
    return L.at(c[0], c[1], c[2]);
  };
  if (kind == LBM_BC_PERIODIC) {
    const int s1 = ((g1 % N) + N) % N, s2 = ((g2 % N) + N) % N;
    const long long d1 = index(g1), d2 = index(g2), r1 = index(s1), r2 = index(s2);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const R v1 = f[i * L.fs + r1], v2 = f[i * L.fs + r2];
      f[i * L.fs + d1] = v1;
      f[i * L.fs + d2] = v2;
    }
    return;
  }
  double G1[5], G2[5];
  if (kind == LBM_BC_FIXED) {
#pragma unroll
    for (int k = 0; k < 5; ++k) G1[k] = G2[k] = bc.fixed[face][k];
  } else {
    double v[NV], M0[5];
    load_cell(f, L.fs, index(hi ? N - 1 : 0), v);
    macros_at(m, v, M0);
    if (kind == LBM_BC_EXTRAPOLATE) {
      double M1[5];
      load_cell(f, L.fs, index(hi ? N - 2 : 1), v);
      macros_at(m, v, M1);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        G1[k] = 2.0 * M0[k] - M1[k];
        G2[k] = 2.0 * G1[k] - M0[k];
      }
    } else {  // LBM_BC_REFLECT
#pragma unroll
      for (int k = 0; k < 5; ++k) G1[k] = G2[k] = M0[k];
      G1[1 + axis] = 0.0;
      G2[1 + axis] = -M0[1 + axis];
    }
  }
  double e[NV];
  equilibrium(m, G1[0], G1[1], G1[2], G1[3], G1[4], e);
  store_cell(f, L.fs, index(g1), e);
  equilibrium(m, G2[0], G2[1], G2[2], G2[3], G2[4], e);
  store_cell(f, L.fs, index(g2), e);
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

constexpr int RED_THREADS = 256;

// Deterministic FP64 sums of (rho, rho u, E) over interior cells: a fixed
// grid-stride assignment, a fixed shared-memory tree per block, and the last
// block to finish adding the per-block partials in block order.
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) conserved_kernel(const R* __restrict__ f, Layout L, Model<double> m,
                                                                double* __restrict__ partials,
                                                                unsigned* __restrict__ counter,
                                                                double* __restrict__ result,
                                                                unsigned* __restrict__ flags) {
  __shared__ double sh[5][RED_THREADS];
  __shared__ bool last;
  double acc[5] = {0, 0, 0, 0, 0};
  bool bad = false;
  const long long n = L.ncell();
  for (long long k = (long long)blockIdx.x * RED_THREADS + threadIdx.x; k < n; k += (long long)gridDim.x * RED_THREADS) {
    int x, y, z;
    cell_of(L, k, x, y, z);
    double v[NV];
    load_cell(f, L.fs, L.at(x, y, z), v);
    const double sa = ((v[1] + v[2]) + (v[3] + v[4])) + (v[5] + v[6]);
    const double sd = ((v[7] + v[8]) + (v[9] + v[10])) + ((v[11] + v[12]) + (v[13] + v[14]));
    const double rho = v[0] + sa + sd;
    const double mx = m.c1 * (v[1] - v[2]) + m.s * (((v[7] + v[8]) + (v[9] + v[10])) - ((v[11] + v[12]) + (v[13] + v[14])));
    const double my = m.c1 * (v[3] - v[4]) + m.s * (((v[7] + v[8]) + (v[11] + v[12])) - ((v[9] + v[10]) + (v[13] + v[14])));
    const double mz = m.c1 * (v[5] - v[6]) + m.s * (((v[7] + v[9]) + (v[11] + v[13])) - ((v[8] + v[10]) + (v[12] + v[14])));
    const double E = m.eta0sq * v[0] + m.c1sq * sa + m.c2sq * sd;
    acc[0] += rho; acc[1] += mx; acc[2] += my; acc[3] += mz; acc[4] += E;
    bad |= !(fabs(rho) + fabs(E) < 1e300);
  }
  if (bad) atomicOr(flags, (unsigned)LBM_HEALTH_NONFINITE);
#pragma unroll
  for (int j = 0; j < 5; ++j) sh[j][threadIdx.x] = acc[j];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int j = 0; j < 5; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < 5; ++j) partials[blockIdx.x * 8 + j] = sh[j][0];
    __threadfence();
    const unsigned done = atomicAdd(counter, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double s[5] = {0, 0, 0, 0, 0};
    for (unsigned b = 0; b < gridDim.x; ++b) {
#pragma unroll
      for (int j = 0; j < 5; ++j) s[j] += ((volatile double*)partials)[b * 8 + j];
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) result[j] = s[j];
    *counter = 0u;
  }
}

inline int blocks_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_fill(int prec, void* f, const Layout& L, const Model<double>& m, const BcDesc& bc, cudaStream_t st) {
  const long long c0 = (long long)L.ny * L.nz, c1 = (long long)L.nx * L.nz, c2 = (long long)L.nx * L.ny;
  long long cmax = c0 > c1 ? c0 : c1;
  cmax = cmax > c2 ? cmax : c2;
  dim3 grid((unsigned)((cmax + 127) / 128), 6);
  if (prec == LBM_FP64) fill_kernel<double><<<grid, 128, 0, st>>>((double*)f, L, m, bc);
  else fill_kernel<float><<<grid, 128, 0, st>>>((float*)f, L, m, bc);
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

cudaError_t launch_conserved(int prec, const void* f, const Layout& L, const Model<double>& m, double* partials,
                             int max_blocks, unsigned* counter, double* result, unsigned* flags, cudaStream_t st) {
  int b = blocks_for(L.ncell(), RED_THREADS);
  if (b > max_blocks) b = max_blocks;
  if (b < 1) b = 1;
  if (prec == LBM_FP64)
    conserved_kernel<double><<<b, RED_THREADS, 0, st>>>((const double*)f, L, m, partials, counter, result, flags);
  else
    conserved_kernel<float><<<b, RED_THREADS, 0, st>>>((const float*)f, L, m, partials, counter, result, flags);
  return cudaGetLastError();
}

}  // namespace lbm
