// Field-split FP32 fused step: two warp groups per 32 x 8 tile.
//
// The tile, the four-plane TMA ring (one 4D copy of all 15 fields per z
// plane, box 40 x 12 x 1 x 15; see tma_ring.cuh) and the per-pair
// arithmetic (pair_math.cuh) are those of the pair kernel.  The CTA has 256
// threads: each of the tile's 128 cell pairs is owned by one thread of group
// 0, which updates f_0 .. f_8 (rest, the six axis velocities and the
// diagonals (+,+,+), (+,+,-)), and by one thread of group 1, which updates
// the six other diagonals.  Both compute the pair's moments (relations
// e1-e3) from all 15 values, so each thread carries the z-marching state
// (planes below, the next plane, the z-interface minmods) of its own fields
// only: about half the registers of the pair kernel, so two CTAs of eight
// warps fit on an SM where the pair kernel fits two of four.  The groups
// split the NND work about evenly (a diagonal velocity has convection along
// three axes, an axis velocity along one plus the dissipation term).
//
// Write-through (WtDesc): each group writes the periodic images of its own
// fields.  The extrapolated / reflected x-face layers need all 15 new values
// of the two boundary cells, so group 0 computes them after the plane's
// barrier, reading group 1's just-stored values back from the output buffer
// (visible to the CTA after the barrier; read through L2).
//
// Every result is bitwise that of the pair kernel.  Measured on the 256^3
// shock-droplet grid (32-plane chunks ending in 8-plane ones): 0.527 ms per
// step against 0.462 for the pair kernel.  Issue efficiency rises from 57 %
// to 62 % with 16 warps per SM, but each group repeats the moments, loads
// the other group's 15 centre values and its own per-plane control work:
// 22 % more instructions, and the groups wait for each other at the plane
// barrier (their NND work differs by about 10 %).
#include "pair_math.cuh"
#include "tma_ring.cuh"

namespace lbm {
namespace {

using pm::ld2;
using ring::mbar_init;
using ring::mbar_expect_tx;
using ring::mbar_wait;
using ring::tma_load_plane;
using ring::tma_prefetch_plane;

struct SplitGeo {
  static constexpr int TX = ring::TX, TY = ring::TY, NSLOT = 4, PF = 2;
  static constexpr int BX = ring::BX, BY = ring::BY, PL = BX * BY;
  static constexpr int SLOT_BYTES = NV * PL * 4;
  static constexpr int SLOT_STRIDE = (SLOT_BYTES + 127) / 128 * 128;
  static constexpr int SMEM = NSLOT * SLOT_STRIDE + NSLOT * 8;
  static constexpr int PAIRS = TX * TY / 2;   // cell pairs of a tile
  static constexpr int THREADS = 2 * PAIRS;   // one thread per pair in each field group
  static constexpr int CTAS_PER_SM = 2;
  static_assert(TX / 2 == 16, "a half warp reads one contiguous tile row");
};

// Fields [lo, hi) of group g.
template <int GROUP>
struct Fields {
  static constexpr int lo = GROUP == 0 ? 0 : 9, hi = GROUP == 0 ? 9 : NV, n = hi - lo;
};

// Barrier 1 over all 256 threads (both groups reach it from their own code),
// with an OR of v across them.
__device__ __forceinline__ bool cta_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((unsigned)v), "n"(SplitGeo::THREADS)
      : "memory");
  return r != 0u;
}
__device__ __forceinline__ void cta_sync() { asm volatile("bar.sync 1, %0;" ::"n"(SplitGeo::THREADS) : "memory"); }

// The x-face layers of plane z for the pair (x, x+1) of row y, which touches
// an extrapolating / reflecting x face: reads the 15 new values of both cells
// from fout (stored by both groups before the barrier) and writes the two
// layers outside the face.
__device__ __noinline__ void split_x_faces(float* __restrict__ fout, const Layout& L, const Model<float>& m,
                                           const WtDesc& wt, int x, int y, int z) {
  const long long g = L.at(x, y, z);
  float a[NV], b[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(fout + i * L.fs + g));
    a[i] = v.x;
    b[i] = v.y;
  }
  const bool lo = x == 0;  // else x == nx - 2
  float g1[NV], g2[NV];
  pm::x_face_layers(m, lo ? wt.xlo : wt.xhi, lo ? a : b, lo ? b : a, g1, g2);
  const long long at = lo ? L.at(-2, y, z) : L.at(L.nx, y, z);
#pragma unroll
  for (int i = 0; i < NV; ++i)
    *reinterpret_cast<float2*>(fout + i * L.fs + at) = lo ? make_float2(g2[i], g1[i]) : make_float2(g1[i], g2[i]);
}

// One z-march unit (the tile column at (x0, y0), planes z0 .. z0+nzc-1) for
// the fields of GROUP.  Both groups call it together (thread 0, in group 0,
// issues the copies); ring plane j is the ring's plane jb + j as in the pair
// kernel.  timed_out is uniform over the CTA.
template <int SCHEME, bool WT, int GROUP>
__device__ __forceinline__ void split_unit(const CUtensorMap* tin, const float* __restrict__ fin,
                                           float* __restrict__ fout, const Layout& L, const Model<float>& m,
                                           const WtDesc& wt, const RecoverDesc& rd, int x0, int y0, int z0, int nzc,
                                           unsigned* __restrict__ flags, unsigned char* smem, uint64_t* bars,
                                           unsigned& jb, bool& timed_out, unsigned wait_limit) {
  using G = SplitGeo;
  using FS = Fields<GROUP>;
  constexpr int NSLOT = G::NSLOT, PL = G::PL, BX = G::BX;
  const int tid = threadIdx.x;
  const int p = tid - GROUP * G::PAIRS;
  const int tx = p % (G::TX / 2), ty = p / (G::TX / 2);
  const int x = x0 + 2 * tx, y = y0 + ty;
  const bool act0 = (x < L.nx) && (y < L.ny);
  const bool act1 = (x + 1 < L.nx) && (y < L.ny);
  const int nplanes = nzc + 2;

  int issued = 0;  // thread 0 only
  auto issue = [&](int j) {
    const unsigned g = jb + (unsigned)j;
    float* dst = reinterpret_cast<float*>(smem + (g % NSLOT) * G::SLOT_STRIDE);
    mbar_expect_tx(&bars[g % NSLOT], G::SLOT_BYTES);
    tma_load_plane(dst, tin, x0 + OX - TMA_LEFT, y0, z0 + j + 2, &bars[g % NSLOT]);
    if (G::PF > 0 && j + G::PF < nplanes) tma_prefetch_plane(tin, x0 + OX - TMA_LEFT, y0, z0 + j + G::PF + 2);
    issued = j + 1;
  };
  if (GROUP == 0 && tid == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int j = 0; j < NSLOT && j < nplanes; ++j) issue(j);
  }
  auto slot = [&](int j) {
    return reinterpret_cast<const float*>(smem + ((jb + (unsigned)j) % NSLOT) * G::SLOT_STRIDE);
  };
  auto arrived = [&](int j) {
    const unsigned g = jb + (unsigned)j;
    return mbar_wait(&bars[g % NSLOT], (g / NSLOT) & 1u, wait_limit);
  };
  auto drained = [&](int j) {
    const unsigned g = jb + (unsigned)j;
    return mbar_wait(&bars[g % NSLOT], (g / NSLOT) & 1u);
  };

  const int c = (ty + 2) * BX + TMA_LEFT + 2 * tx;
  const long long gbase = L.at(x, y, z0);

  float2 h1[FS::n], h2[FS::n], carry[FS::n];
#pragma unroll
  for (int j = 0; j < FS::n; ++j) {
    const int i = FS::lo + j;
    h1[j] = act0 ? ld2(fin + i * L.fs + gbase - L.plane) : make_float2(0.f, 0.f);
    h2[j] = act0 ? ld2(fin + i * L.fs + gbase - 2 * L.plane) : make_float2(0.f, 0.f);
    carry[j] = make_float2(0.f, 0.f);
  }

  unsigned bad = 0u;
  {
    bool ok = true;
    for (int j = 0; j < 3; ++j) ok = arrived(j) && ok;
    timed_out = cta_sync_or(!ok);
  }
  if (!timed_out && SCHEME == LBM_SCHEME_NND) {
    const float* P0 = slot(0);
    const float* P1 = slot(1);
#pragma unroll
    for (int j = 0; j < FS::n; ++j) {
      const int i = FS::lo + j;
      carry[j] = pm::carry0(i, h2[j], h1[j], ld2(P0 + i * PL + c), ld2(P1 + i * PL + c));
    }
  }

  float2 F[FS::n], Fn[FS::n];
  if (!timed_out) {
    const float* Q0 = slot(0);
#pragma unroll
    for (int j = 0; j < FS::n; ++j) F[j] = ld2(Q0 + (FS::lo + j) * PL + c);
  }
  for (int k = 0; k < nzc && !timed_out; ++k) {
    const float* P0 = slot(k);
    const float* P1 = slot(k + 1);
    const float* P2 = slot(k + 2);

    // all 15 values of the pair: this group's from registers, the other's from the plane tile
    float2 V[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) V[i] = (i >= FS::lo && i < FS::hi) ? F[i - FS::lo] : ld2(P0 + i * PL + c);
    const pm::Mom r = pm::moments(m, rd, V, P0, c, PL, act0, act1);
    if (GROUP == 0) bad |= pm::health(r, act0, act1);
    float2 out[FS::n];
#pragma unroll
    for (int j = 0; j < FS::n; ++j) {
      const int i = FS::lo + j;
      const float2 Z1 = ld2(P1 + i * PL + c);
      Fn[j] = Z1;
      float2 unused;
      out[j] = pm::field_update<SCHEME, BX>(m, i, P0 + i * PL + c, F[j], Z1, P2 + i * PL + c, h1[j], h2[j],
                                            carry[j], unused, pm::feq(m, r, i));
    }
    const long long g = gbase + (long long)k * L.plane;
    if (act1) {
#pragma unroll
      for (int j = 0; j < FS::n; ++j) *reinterpret_cast<float2*>(fout + (FS::lo + j) * L.fs + g) = out[j];
    } else if (act0) {
#pragma unroll
      for (int j = 0; j < FS::n; ++j) fout[(FS::lo + j) * L.fs + g] = out[j].x;
    }
    // periodic images of this group's fields (at most one per axis)
    if (WT && act0) {
      const int z = z0 + k;
      long long ay = -1, az = -1, ax = -1;
      if (wt.per[1]) ay = y < 2 ? L.at(x, y + L.ny, z) : (y >= L.ny - 2 ? L.at(x, y - L.ny, z) : -1);
      if (wt.per[2]) az = z < 2 ? L.at(x, y, z + L.nz) : (z >= L.nz - 2 ? L.at(x, y, z - L.nz) : -1);
      if (wt.per[0]) ax = x == 0 ? L.at(L.nx, y, z) : (x == L.nx - 2 ? L.at(-2, y, z) : -1);
      if (ay >= 0 || az >= 0 || ax >= 0) {
#pragma unroll 1
        for (int q = 0; q < 3; ++q) {
          const long long at = q == 0 ? ay : (q == 1 ? az : ax);
          if (at < 0) continue;
          if (act1) {
#pragma unroll
            for (int j = 0; j < FS::n; ++j) *reinterpret_cast<float2*>(fout + (FS::lo + j) * L.fs + at) = out[j];
          } else {
#pragma unroll
            for (int j = 0; j < FS::n; ++j) fout[(FS::lo + j) * L.fs + at] = out[j].x;
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < FS::n; ++j) {
      h2[j] = h1[j];
      h1[j] = F[j];
      F[j] = Fn[j];
    }
    // ring plane k+3 must have landed; the barrier also retires plane k, whose slot takes plane k + NSLOT
    const bool ok = (k + 3 < nplanes) ? arrived(k + 3) : true;
    if (cta_sync_or(!ok)) {
      timed_out = true;
      break;
    }
    if (GROUP == 0 && tid == 0 && k + NSLOT < nplanes) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(k + NSLOT);
    }
    // x-face layers of the plane just finished (both groups' values are in fout)
    if (WT && GROUP == 0 && act1 && ((wt.xlo && x == 0) || (wt.xhi && x == L.nx - 2)))
      split_x_faces(fout, L, m, wt, x, y, z0 + k);
  }

  if (tid == 0 && timed_out) atomicOr(flags, (unsigned)LBM_HEALTH_TIMEOUT);
  if (bad) atomicOr(flags, bad);
  if (timed_out) {
    // leave no copy in flight: the newest plane of each slot is waited for (bounded)
    if (tid == 0)
      for (int j = max(0, issued - NSLOT); j < issued; ++j) drained(j);
    cta_sync();
  }
  jb += (unsigned)nplanes;
}

template <int SCHEME, bool WT>
__global__ void __launch_bounds__(SplitGeo::THREADS, SplitGeo::CTAS_PER_SM)
    step_split_kernel(const __grid_constant__ CUtensorMap tin, const float* __restrict__ fin,
                      float* __restrict__ fout, Layout L, Model<float> m, WtDesc wt, RecoverDesc rd, ZSched zs,
                      unsigned* __restrict__ flags, unsigned wait_limit) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SplitGeo::NSLOT * SplitGeo::SLOT_STRIDE);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < SplitGeo::NSLOT; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned jb = 0;
  bool timed_out = false;
  const int x0 = blockIdx.x * SplitGeo::TX, y0 = blockIdx.y * SplitGeo::TY;
  const int z0 = zs.z0(blockIdx.z), nzc = zs.len(blockIdx.z, L.nz);
  if (threadIdx.x < SplitGeo::PAIRS)
    split_unit<SCHEME, WT, 0>(&tin, fin, fout, L, m, wt, rd, x0, y0, z0, nzc, flags, smem, bars, jb, timed_out,
                              wait_limit);
  else
    split_unit<SCHEME, WT, 1>(&tin, fin, fout, L, m, wt, rd, x0, y0, z0, nzc, flags, smem, bars, jb, timed_out,
                              wait_limit);
}

// Persistent batched form (the pair kernel's work queue over the descriptor
// table; see step_pair_batch_kernel).
template <int SCHEME>
__global__ void __launch_bounds__(SplitGeo::THREADS, SplitGeo::CTAS_PER_SM)
    step_split_batch_kernel(const __grid_constant__ BatchTable tab) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SplitGeo::NSLOT * SplitGeo::SLOT_STRIDE);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < SplitGeo::NSLOT; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned jb = 0;
  bool timed_out = false;
  __shared__ long long next;
  for (;;) {
    if (threadIdx.x == 0) next = (long long)atomicAdd(tab.queue, 1ull);
    __syncthreads();
    const long long u = next;
    __syncthreads();
    if (u >= tab.total_units || timed_out) break;
    int e = 0;
    while (e + 1 < tab.n && u >= tab.item[e + 1].first_unit) ++e;
    const BatchItem& it = tab.item[e];
    const long long local = u - it.first_unit;
    const long long per_chunk = (long long)it.tiles_x * it.tiles_y;
    const int chunk = (int)(local / per_chunk);
    const int t = (int)(local % per_chunk);
    // the unit's descriptors as locals (see step_pair_batch_kernel)
    const Layout L = it.L;
    const Model<float> m = it.m;
    const WtDesc wt = it.wt;
    const RecoverDesc rd = it.rd;
    const ZSched zs = it.zs;
    const int x0 = (t % it.tiles_x) * SplitGeo::TX, y0 = (t / it.tiles_x) * SplitGeo::TY;
    if (threadIdx.x < SplitGeo::PAIRS)
      split_unit<SCHEME, true, 0>(&tab.map[e], it.fin, it.fout, L, m, wt, rd, x0, y0, zs.z0(chunk),
                                  zs.len(chunk, L.nz), it.flags, smem, bars, jb, timed_out, tab.wait_limit);
    else
      split_unit<SCHEME, true, 1>(&tab.map[e], it.fin, it.fout, L, m, wt, rd, x0, y0, zs.z0(chunk),
                                  zs.len(chunk, L.nz), it.flags, smem, bars, jb, timed_out, tab.wait_limit);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(tab.done, 1u) == gridDim.x - 1) {
      *tab.queue = 0ull;
      *tab.done = 0u;
      __threadfence();
    }
  }
}

template <int SCHEME>
cudaError_t set_split_attributes() {
  cudaError_t e = cudaFuncSetAttribute(step_split_kernel<SCHEME, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SplitGeo::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_split_kernel<SCHEME, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SplitGeo::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_split_batch_kernel<SCHEME>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SplitGeo::SMEM);
  return e;
}

template <int SCHEME>
void launch_split_scheme(const CUtensorMap& map, const float* fin, float* fout, const Layout& L,
                         const Model<float>& m, const WtDesc& wt, const RecoverDesc& rd, const ZSched& zs,
                         unsigned* flags, unsigned wait_limit, cudaStream_t st) {
  dim3 grid((L.nx + SplitGeo::TX - 1) / SplitGeo::TX, (L.ny + SplitGeo::TY - 1) / SplitGeo::TY, zs.nch);
  const bool any = wt.per[0] || wt.per[1] || wt.per[2] || wt.xlo || wt.xhi;
  if (any)
    step_split_kernel<SCHEME, true><<<grid, SplitGeo::THREADS, SplitGeo::SMEM, st>>>(map, fin, fout, L, m, wt, rd,
                                                                                     zs, flags, wait_limit);
  else
    step_split_kernel<SCHEME, false><<<grid, SplitGeo::THREADS, SplitGeo::SMEM, st>>>(map, fin, fout, L, m, wt, rd,
                                                                                      zs, flags, wait_limit);
}

}  // namespace

cudaError_t prepare_split_kernels() {
  cudaError_t e = set_split_attributes<LBM_SCHEME_NND>();
  if (e == cudaSuccess) e = set_split_attributes<LBM_SCHEME_UPWIND2>();
  if (e == cudaSuccess) e = set_split_attributes<LBM_SCHEME_UPWIND1>();
  return e;
}

cudaError_t launch_step_split(int scheme, const CUtensorMap& map, const float* fin, float* fout, const Layout& L,
                              const Model<float>& m, const WtDesc& wt, const RecoverDesc& rd, const ZSched& zs,
                              unsigned* flags, unsigned wait_limit, cudaStream_t st) {
  switch (scheme) {
    case LBM_SCHEME_NND: launch_split_scheme<LBM_SCHEME_NND>(map, fin, fout, L, m, wt, rd, zs, flags, wait_limit, st); break;
    case LBM_SCHEME_UPWIND2:
      launch_split_scheme<LBM_SCHEME_UPWIND2>(map, fin, fout, L, m, wt, rd, zs, flags, wait_limit, st);
      break;
    default: launch_split_scheme<LBM_SCHEME_UPWIND1>(map, fin, fout, L, m, wt, rd, zs, flags, wait_limit, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_step_split_batch(int scheme, const BatchTable& tab, int grid, cudaStream_t st) {
  switch (scheme) {
    case LBM_SCHEME_NND:
      step_split_batch_kernel<LBM_SCHEME_NND><<<grid, SplitGeo::THREADS, SplitGeo::SMEM, st>>>(tab);
      break;
    case LBM_SCHEME_UPWIND2:
      step_split_batch_kernel<LBM_SCHEME_UPWIND2><<<grid, SplitGeo::THREADS, SplitGeo::SMEM, st>>>(tab);
      break;
    default: step_split_batch_kernel<LBM_SCHEME_UPWIND1><<<grid, SplitGeo::THREADS, SplitGeo::SMEM, st>>>(tab);
  }
  return cudaGetLastError();
}

}  // namespace lbm
