// Tiled single-precision fused step for sm_103a.
//
// A CTA owns a TX x TY column of cells and marches it through a chunk of z
// planes.  Each plane of all 15 fields, with a two-cell halo in x and y, is
// brought into shared memory by one 4D TMA copy (box 36 x 12 x 1 x 15) into a
// ring of NSLOT slots; completion is tracked by one mbarrier per slot, and the
// copy for plane z+NSLOT is issued as soon as plane z is retired, so a full
// step of compute hides each copy.  Per cell the kernel forms the moments,
// the equilibrium (Eq. "eq"), the NND differences along x and y from the
// shared tile and along z from the plane ring, the lambda_i Laplacian
// (Eq. "lp"), and writes the BGK / forward-Euler update to global memory.
//
// The minmod of the interface between planes z and z+1 is computed once: it
// is carried in a register from plane z to plane z+1 (the NND flux of that
// interface is shared by the two cells it separates).
//
// Every wait on an mbarrier is bounded; on timeout the CTA sets
// LBM_HEALTH_TIMEOUT in the status word, waits (bounded) for its own copies in
// flight and returns.
#include "tma_ring.cuh"

namespace lbm {
namespace {

using namespace ring;

template <int SCHEME>
__global__ void __launch_bounds__(TX* TY, 2)
    step_tiled_kernel(const __grid_constant__ CUtensorMap tin, const float* __restrict__ fin, float* __restrict__ fout,
                      Layout L, Model<float> m, int zc, unsigned* __restrict__ flags) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NSLOT * SLOT_STRIDE);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * zc;
  const int nzc = min(zc, L.nz - z0);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = (x < L.nx) && (y < L.ny);
  const int nplanes = nzc + 2;  // planes z0 .. z0+nzc+1 pass through the ring

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  // plane j (interior z0 + j, padded z0 + j + 2) goes to slot j % NSLOT
  int issued = 0;  // meaningful in thread 0 only
  auto issue = [&](int j) {
    const int s = j % NSLOT;
    float* dst = reinterpret_cast<float*>(smem + s * SLOT_STRIDE);
    mbar_expect_tx(&bars[s], SLOT_BYTES_TX);
    tma_load_plane(dst, &tin, x0 + OX - TMA_LEFT, y0, z0 + j + 2, &bars[s]);
    issued = j + 1;
  };
  if (tid == 0) {
    for (int j = 0; j < NSLOT && j < nplanes; ++j) issue(j);
  }
  auto slot = [&](int j) { return reinterpret_cast<const float*>(smem + (j % NSLOT) * SLOT_STRIDE); };
  // all threads poll (bounded); the outcome is made uniform by the barrier
  auto landed = [&](int j) {
    const bool ok = mbar_wait(&bars[j % NSLOT], (unsigned)((j / NSLOT) & 1));
    return __syncthreads_or(!ok) == 0;
  };

  const int c = (ty + 2) * BX + (tx + TMA_LEFT);
  const long long gbase = L.at(x, y, z0);

  // own column one and two planes below z0 (ghost planes when z0 = 0)
  float h1[NV], h2[NV], carry[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    h1[i] = active ? fin[i * L.fs + gbase - L.plane] : 0.f;
    h2[i] = active ? fin[i * L.fs + gbase - 2 * L.plane] : 0.f;
    carry[i] = 0.f;
  }

  unsigned bad = 0u;
  bool timed_out = !landed(0) || !landed(1);
  if (!timed_out && SCHEME == LBM_SCHEME_NND) {
    // minmod of the interface below plane z0 (carried upward from then on)
    const float* P0 = slot(0);
    const float* P1 = slot(1);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int sz = vsign(i, 2);
      const float fc = P0[i * PL + c];
      if (sz > 0) carry[i] = minmod(fc - h1[i], h1[i] - h2[i]);
      if (sz < 0) carry[i] = minmod(fc - h1[i], P1[i * PL + c] - fc);
    }
  }

  for (int k = 0; k < nzc && !timed_out; ++k) {
    if (!landed(k + 2)) {
      timed_out = true;
      break;
    }
    const float* P0 = slot(k);
    const float* P1 = slot(k + 1);
    const float* P2 = slot(k + 2);

    float f[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) f[i] = P0[i * PL + c];

    float rho, ux, uy, uz, T;
    moments(m, f, rho, ux, uy, uz, T);
    if (active) {
      if (!(rho > 0.f)) bad |= LBM_HEALTH_RHO;
      if (!(T > 0.f)) bad |= LBM_HEALTH_T;
      if (!(fabsf(rho) + fabsf(T) + fabsf(ux) + fabsf(uy) + fabsf(uz) < 1e30f)) bad |= LBM_HEALTH_NONFINITE;
    }
    float feq[NV];
    equilibrium(m, rho, ux, uy, uz, T, feq);

    float out[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float* q = P0 + i * PL + c;
      const float fc = f[i];
      float conv = 0.f, lap = 0.f;
      // x
      {
        const int sg = vsign(i, 0);
        if (sg > 0) {
          const float m1 = q[-1], p1 = q[1];
          conv += grad_pos<SCHEME>(q[-2], m1, fc, p1);
          if (i <= 6) lap += (p1 - 2.f * fc) + m1;
        } else if (sg < 0) {
          const float m1 = q[-1], p1 = q[1];
          conv -= grad_neg<SCHEME>(m1, fc, p1, q[2]);
          if (i <= 6) lap += (p1 - 2.f * fc) + m1;
        } else if (i <= 6) {
          lap += (q[1] - 2.f * fc) + q[-1];
        }
      }
      // y
      {
        const int sg = vsign(i, 1);
        if (sg > 0) {
          const float m1 = q[-BX], p1 = q[BX];
          conv += grad_pos<SCHEME>(q[-2 * BX], m1, fc, p1);
          if (i <= 6) lap += (p1 - 2.f * fc) + m1;
        } else if (sg < 0) {
          const float m1 = q[-BX], p1 = q[BX];
          conv -= grad_neg<SCHEME>(m1, fc, p1, q[2 * BX]);
          if (i <= 6) lap += (p1 - 2.f * fc) + m1;
        } else if (i <= 6) {
          lap += (q[BX] - 2.f * fc) + q[-BX];
        }
      }
      // z: the ring holds planes z+1 and z+2, registers hold z-1 (and z-2)
      {
        const int sg = vsign(i, 2);
        const float p1 = P1[i * PL + c];
        const float m1 = h1[i];
        if (sg > 0) {
          float G;
          if (SCHEME == LBM_SCHEME_NND) {
            const float d0 = fc - m1;
            const float mmA = minmod(p1 - fc, d0);
            G = d0 + 0.5f * (mmA - carry[i]);
            carry[i] = mmA;
          } else {
            G = grad_pos<SCHEME>(h2[i], m1, fc, p1);
          }
          conv += G;
        } else if (sg < 0) {
          const float p2 = P2[i * PL + c];
          float G;
          if (SCHEME == LBM_SCHEME_NND) {
            const float d1 = p1 - fc;
            const float mmC = minmod(d1, p2 - p1);
            G = d1 - 0.5f * (mmC - carry[i]);
            carry[i] = mmC;
          } else {
            G = grad_neg<SCHEME>(m1, fc, p1, p2);
          }
          conv -= G;
        }
        if (i <= 6) lap += (p1 - 2.f * fc) + m1;
      }
      const float kk = i == 0 ? 0.f : (i <= 6 ? m.k1 : m.k2);
      const float lam = i == 0 ? m.lam0 : (i <= 6 ? m.lam1 : 0.f);
      out[i] = fc + m.dt_tau * (feq[i] - fc) - kk * conv + lam * lap;
    }
    if (active) {
      const long long g = gbase + (long long)k * L.plane;
#pragma unroll
      for (int i = 0; i < NV; ++i) fout[i * L.fs + g] = out[i];
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      h2[i] = h1[i];
      h1[i] = f[i];
    }
    // every thread is done with plane k: its slot takes plane k + NSLOT
    __syncthreads();
    if (tid == 0 && k + NSLOT < nplanes) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(k + NSLOT);
    }
  }

  if (tid == 0 && timed_out) atomicOr(flags, (unsigned)LBM_HEALTH_TIMEOUT);
  if (bad) atomicOr(flags, bad);
  // leave no copy in flight: the newest plane of each slot is waited for (bounded)
  if (tid == 0) {
    for (int j = max(0, issued - NSLOT); j < issued; ++j) mbar_wait(&bars[j % NSLOT], (unsigned)((j / NSLOT) & 1));
  }
  __syncthreads();
}

template <int SCHEME>
cudaError_t launch_scheme(const CUtensorMap& map, const float* fin, float* fout, const Layout& L,
                          const Model<float>& m, int zc, unsigned* flags, cudaStream_t st) {
  dim3 block(TX, TY, 1);
  dim3 grid((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY, (L.nz + zc - 1) / zc);
  step_tiled_kernel<SCHEME><<<grid, block, SMEM_BYTES, st>>>(map, fin, fout, L, m, zc, flags);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_tiled_kernels() {
  cudaError_t e = cudaFuncSetAttribute(step_tiled_kernel<LBM_SCHEME_NND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_tiled_kernel<LBM_SCHEME_UPWIND2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_tiled_kernel<LBM_SCHEME_UPWIND1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SMEM_BYTES);
  return e;
}

int tiled_box_x() { return BX; }
int tiled_box_y() { return BY; }

cudaError_t launch_step_tiled(int scheme, const CUtensorMap& map, const float* fin, float* fout, const Layout& L,
                              const Model<float>& m, int zc, unsigned* flags, cudaStream_t st) {
  switch (scheme) {
    case LBM_SCHEME_NND: return launch_scheme<LBM_SCHEME_NND>(map, fin, fout, L, m, zc, flags, st);
    case LBM_SCHEME_UPWIND2: return launch_scheme<LBM_SCHEME_UPWIND2>(map, fin, fout, L, m, zc, flags, st);
    default: return launch_scheme<LBM_SCHEME_UPWIND1>(map, fin, fout, L, m, zc, flags, st);
  }
}

}  // namespace lbm
