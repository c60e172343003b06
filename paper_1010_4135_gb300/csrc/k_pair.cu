// Tiled single-precision fused step, two x-adjacent cells per thread.
//
// Same plane ring as step_tiled_kernel (one 4D TMA copy per z plane into an
// mbarrier-tracked ring; see tma_ring.cuh), but each thread of a TX x 8 tile
// (PairGeo below; 32 x 8 and 128 threads by default) owns the cell pair
// (x, x+1).  The pair is loaded with one
// 64-bit shared load per field and neighbour row, and everything that is the
// same arithmetic for both cells runs as packed f32x2 operations (FADD2,
// FMUL2, FFMA2), which halves the instructions the schedulers issue.
//
// Per interface the NND minmod is evaluated once: minmod(x, d) is x clamped
// to [min(d, 0), max(d, 0)], the two minmods of one cell share d, the pair
// shares the minmod of its middle x-interface, and the minmod of each
// z-interface is carried from plane z to plane z+1.  The Laplacian centre
// and the relaxation are folded into one coefficient per velocity shell:
//   f_new = keep_i f + (dt/tau) f^eq - (|v| dt/dx) C + (lambda_i dt/dx^2) S,
// with S the sum of the six neighbours and keep_i = 1 - dt/tau - 6 lambda_i dt/dx^2.
//
// The kernel also writes the boundary layers of the state it produces
// (WtDesc): periodic images of the first and last two rows, planes and (for
// even nx) columns, and the x-face layers of extrapolating or reflecting
// faces (Sec. 4(2) rules applied to the two new boundary cells, which the
// same thread holds), so the next step needs no separate fill for them.
#include "pair_math.cuh"
#include "tma_ring.cuh"

namespace lbm {
namespace {

using ring::mbar_init;
using ring::mbar_expect_tx;
using ring::mbar_wait;
using ring::tma_load_plane;
using ring::tma_prefetch_plane;

// Tile geometry of the pair kernel: a TX x TY column of cells, one thread per
// cell pair (x, x+1), and a four-plane ring: cell plane z reads ring planes z
// (its x / y neighbours), z+1 and z+2 while z+3 lands.  PF > 0 also asks the
// TMA unit to bring ring plane j+PF into L2 when plane j is copied, which
// keeps more DRAM reads in flight per SM than the ring alone.
template <int TX_, int TY_, int PF_, bool SPLIT_ = false>
struct PairGeo {
  static constexpr int TX = TX_, TY = TY_, NSLOT = 4, PF = PF_;
  // SPLIT: the CTA works as two independent halves of 128 threads (the left
  // and right 32 x 8 cells), each with its own named barrier per plane; a
  // slot is refilled by whichever half releases it second (release counters
  // after the mbarriers), so one half can run a plane ahead of the other.
  static constexpr bool SPLIT = SPLIT_;
  static constexpr int BX = TX + 2 * TMA_LEFT, BY = TY + 4;  // tile with its halo
  static constexpr int PL = BX * BY;                          // floats per field in one plane tile
  static constexpr int SLOT_BYTES = NV * PL * 4;              // bytes one TMA copy delivers
  static constexpr int SLOT_STRIDE = (SLOT_BYTES + 127) / 128 * 128;
  // slots, then the mbarriers, then (SPLIT) the release counters and the issued-plane count
  static constexpr int SMEM = NSLOT * SLOT_STRIDE + NSLOT * 8 + (SPLIT ? 64 : 0);
  static constexpr int PX = TX / 2;                           // threads along x
  static constexpr int THREADS = PX * TY;
  // CTAs per SM that the shared memory allows (228 KB per SM, 1 KB reserved
  // per CTA, the batched kernel's 8-byte work-queue slot rounded to 128)
  static constexpr int CTAS_PER_SM = 233472 / (SMEM + 128 + 1024);
  static_assert(CTAS_PER_SM >= 1, "ring fits one CTA");
  static_assert(THREADS % 32 == 0, "whole warps");
  static_assert(PX == 16 || PX == 32,
                "64-bit shared loads: a half warp (one 128-byte wavefront) reads one contiguous tile row");
  static_assert(BX * 4 % 16 == 0 && BX <= 256, "TMA box inner extent: a 16-byte multiple, at most 256");
  static_assert(TX % 32 == 0, "tile rows start on 32-byte sectors (OX is a multiple of 8)");
  static_assert(!SPLIT || (PX == 32 && TY == 8), "split halves: 16 pairs x 8 rows of 128 threads each");
  // SPLIT: thread t of half h = t / 128 owns pair column 16 h + t % 16 of row (t % 128) / 16
  __device__ static int col(int tid) { return SPLIT ? (tid & 15) + 16 * (tid >> 7) : tid % PX; }
  __device__ static int row(int tid) { return SPLIT ? (tid & 127) >> 4 : tid / PX; }
};
// 32 x 8 tiles (the single-cell tiled kernel's box, 40 x 12): two CTAs of 4
// warps per SM, L2 prefetch two planes ahead (256^3: 0.475 ms per step, 0.488
// without the prefetch; one or three planes ahead: no faster).
using Geo32 = PairGeo<ring::TX, ring::TY, 2>;
// 64 x 8 tiles (box 72 x 12 x 1 x 15): one CTA of 8 warps per SM, 288-byte
// row reads, run as two split halves.  Its data movement alone (ring +
// stores, no arithmetic) is faster (0.362 ms against 0.443 ms on 256^3);
// with the arithmetic it takes 0.511 ms (0.549 ms with one CTA-wide barrier
// per plane), against 0.465 ms for two independent 32 x 8 CTAs per SM.
using Geo64 = PairGeo<64, 8, 2, true>;
static_assert(Geo32::BX == ring::BX && Geo32::BY == ring::BY, "Geo32 shares the tiled kernel's tensor map");

using pm::bc2;
using pm::ld2;

// Named barrier `id` over 128 threads with an OR of v across them.
__device__ __forceinline__ bool half_sync_or(unsigned id, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((unsigned)v), "r"(id)
      : "memory");
  return r != 0u;
}

// One z-march unit: the TX x TY column at (x0, y0), planes z0 .. z0+nzc-1.
// Plane j of the unit is the ring's plane number jb + j (slot (jb+j) % NSLOT,
// phase parity ((jb+j) / NSLOT) & 1), so consecutive units of a CTA keep
// using the same barriers; jb advances by the unit's plane count.  All
// threads of the CTA call it together; timed_out is uniform.  FULL: every
// tile lies inside the grid (nx and ny multiples of the tile), so every pair
// is active and the activity tests fold away.
template <int SCHEME, bool WT, class G, bool FULL = false, bool R1 = false>
__device__ __forceinline__ void pair_unit(const CUtensorMap* tin, const float* __restrict__ fin,
                                          float* __restrict__ fout, const Layout& L, const Model<float>& m,
                                          const WtDesc& wt, const RecoverDesc& rd, int x0, int y0, int z0,
                                          int nzc,
                                          unsigned* __restrict__ flags, unsigned char* smem, uint64_t* bars,
                                          unsigned& jb, bool& timed_out, unsigned wait_limit) {
  constexpr int NSLOT = G::NSLOT, PL = G::PL, BX = G::BX;
  const int tid = threadIdx.x;
  const int tx = G::col(tid), ty = G::row(tid);
  const int x = x0 + 2 * tx, y = y0 + ty;
  const bool act0 = FULL || ((x < L.nx) && (y < L.ny));
  const bool act1 = FULL || ((x + 1 < L.nx) && (y < L.ny));
  // ring planes 0 .. nzc+1 are the padded planes z0+2 .. z0+nzc+3 (interior
  // z0 .. z0+nzc+1); cell plane k reads ring planes k, k+1, k+2
  const int nplanes = nzc + 2;

  // copy ring plane j (interior z0 + j, padded z0 + j + 2) into its slot
  // (SPLIT: release counters and the count of issued planes follow the mbarriers)
  unsigned* rel = reinterpret_cast<unsigned*>(bars + NSLOT);
  int* issued_s = reinterpret_cast<int*>(rel + NSLOT);
  int issued = 0;  // thread 0 only (without SPLIT)
  auto issue = [&](int j) {
    const unsigned g = jb + (unsigned)j;
    float* dst = reinterpret_cast<float*>(smem + (g % NSLOT) * G::SLOT_STRIDE);
    mbar_expect_tx(&bars[g % NSLOT], G::SLOT_BYTES);
    tma_load_plane(dst, tin, x0 + OX - TMA_LEFT, y0, z0 + j + 2, &bars[g % NSLOT]);
    if (G::PF > 0 && j + G::PF < nplanes) tma_prefetch_plane(tin, x0 + OX - TMA_LEFT, y0, z0 + j + G::PF + 2);
    if (G::SPLIT) atomicMax(issued_s, j + 1);
    else issued = j + 1;
  };
  if (tid == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (G::SPLIT) *issued_s = 0;
    for (int j = 0; j < NSLOT && j < nplanes; ++j) issue(j);
  }
  auto slot = [&](int j) {
    return reinterpret_cast<const float*>(smem + ((jb + (unsigned)j) % NSLOT) * G::SLOT_STRIDE);
  };
  // waits for data use wait_limit; the drain after a timeout uses the full limit
  auto arrived = [&](int j) {
    const unsigned g = jb + (unsigned)j;
    return mbar_wait(&bars[g % NSLOT], (g / NSLOT) & 1u, wait_limit);
  };
  auto drained = [&](int j) {
    const unsigned g = jb + (unsigned)j;
    return mbar_wait(&bars[g % NSLOT], (g / NSLOT) & 1u);
  };

  const int c = (ty + 2) * BX + TMA_LEFT + 2 * tx;  // own pair in a plane tile (even: 8-byte aligned)
  const long long gbase = L.at(x, y, z0);

  float2 h1[NV], h2[NV], carry[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    h1[i] = act0 ? ld2(fin + i * L.fs + gbase - L.plane) : make_float2(0.f, 0.f);
    h2[i] = act0 ? ld2(fin + i * L.fs + gbase - 2 * L.plane) : make_float2(0.f, 0.f);
    carry[i] = make_float2(0.f, 0.f);
  }

  unsigned bad = 0u;
  // ring planes 0 .. 2 must have landed; the outcome is made uniform by the barrier
  {
    bool ok = true;
    for (int j = 0; j < 3; ++j) ok = arrived(j) && ok;
    timed_out = __syncthreads_or(!ok) != 0;
  }
  if (!timed_out && SCHEME == LBM_SCHEME_NND) {
    const float* P0 = slot(0);
    const float* P1 = slot(1);
#pragma unroll
    for (int i = 0; i < NV; ++i) carry[i] = pm::carry0(i, h2[i], h1[i], ld2(P0 + i * PL + c), ld2(P1 + i * PL + c));
  }

  // Besides the own pair of plane k (F, below), the planes below are carried
  // in registers only where a field needs them: h1 for the Laplacian of
  // f_0..f_6 and the z stencil of the axis velocities, the lower z difference
  // (dz) for the diagonal velocities with v_z > 0 (NND), and h2 for the
  // second-order upwind scheme.
  constexpr bool DZ = SCHEME == LBM_SCHEME_NND;
  float2 dz[NV];
  if (!timed_out && DZ) {
    const float* Q0 = slot(0);
#pragma unroll
    for (int i = 7; i < NV; ++i)
      if (vsign(i, 2) > 0) dz[i] = pm::sub(ld2(Q0 + i * PL + c), h1[i]);
  }
  // health: running minima of rho and T and a running sum of rho + T of each
  // cell of the pair, judged once at the end of the unit.  A non-finite rho or
  // T makes the sum non-finite, and so does a non-finite velocity: T is
  // (E/rho - u^2)/b, -inf or NaN when u^2 is inf or NaN.
  float2 hmin_rho = make_float2(INFINITY, INFINITY), hmin_T = hmin_rho, hsum = make_float2(0.f, 0.f);
  // write-through targets that do not depend on the plane: the periodic y and
  // x images of this pair (element offsets from its own index, 0 = none)
  long long img_y = 0, img_x = 0;
  if (WT && act0) {
    if (wt.per[1]) img_y = y < 2 ? (long long)L.ny * L.sx : (y >= L.ny - 2 ? -(long long)L.ny * L.sx : 0);
    if (wt.per[0]) img_x = x == 0 ? L.nx : (x == L.nx - 2 ? -L.nx : 0);
  }
  const bool face_lo = WT && act0 && wt.xlo && x == 0, face_hi = WT && act0 && wt.xhi && x == L.nx - 2;
  // the pair's own values of the plane: loaded once for the first plane, then
  // carried from the previous plane's z-neighbour loads, so that the moments
  // of a plane start without waiting on shared memory (256^3: 0.4206 ->
  // 0.4173 ms per step, although the register rotation adds instructions)
  float2 F[NV];
  if (!timed_out) {
    const float* Q0 = slot(0);
#pragma unroll
    for (int i = 0; i < NV; ++i) F[i] = ld2(Q0 + i * PL + c);
  }
  for (int k = 0; k < nzc && !timed_out; ++k) {
    const float* P0 = slot(k);
    const float* P1 = slot(k + 1);
    const float* P2 = slot(k + 2);
    float2 Z1[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) Z1[i] = ld2(P1 + i * PL + c);

    // moments (relations e1-e3), health, equilibrium and the per-field update
    const pm::Mom r = pm::moments(m, rd, F, P0, c, PL, act0, act1);
    hmin_rho = make_float2(fminf(hmin_rho.x, r.rho.x), fminf(hmin_rho.y, r.rho.y));
    hmin_T = make_float2(fminf(hmin_T.x, r.T.x), fminf(hmin_T.y, r.T.y));
    hsum = pm::add(hsum, pm::add(r.rho, r.T));
    float2 out[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      out[i] = pm::field_update<SCHEME, BX, DZ, R1>(m, i, P0 + i * PL + c, F[i], Z1[i], P2 + i * PL + c,
                                                h1[i], h2[i], carry[i], dz[i], pm::feq(m, r, i));
    // the pair's element offset within a field: below 2^32 (the host rejects
    // longer fields), so the fields' stores share one 32-bit offset
    const unsigned g = (unsigned)gbase + (unsigned)k * (unsigned)L.plane;
    if (act1) {
#pragma unroll
      for (int i = 0; i < NV; ++i) *reinterpret_cast<float2*>(fout + i * L.fs + g) = out[i];
    } else if (act0) {
#pragma unroll
      for (int i = 0; i < NV; ++i) fout[i * L.fs + g] = out[i].x;
    }
    // ---- boundary layers of the new state (write-through): at most one
    // periodic image per axis (axes of >= 4 cells), and the x-face layers
    if (WT && act0) {
      const int z = z0 + k;
      long long img_z = 0;
      if (wt.per[2]) img_z = z < 2 ? (long long)L.nz * L.plane : (z >= L.nz - 2 ? -(long long)L.nz * L.plane : 0);
      if (img_y | img_z | img_x) {
#pragma unroll 1
        for (int q = 0; q < 3; ++q) {
          const long long off = q == 0 ? img_y : (q == 1 ? img_z : img_x);
          if (off == 0) continue;
          const long long at = (long long)g + off;
          if (act1) {
#pragma unroll
            for (int i = 0; i < NV; ++i) *reinterpret_cast<float2*>(fout + i * L.fs + at) = out[i];
          } else {
#pragma unroll
            for (int i = 0; i < NV; ++i) fout[i * L.fs + at] = out[i].x;
          }
        }
      }
      if (face_lo || face_hi) {
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
          if (side == 0 ? !face_lo : !face_hi) continue;
          float c0[NV], c1[NV], g1[NV], g2[NV];
#pragma unroll
          for (int i = 0; i < NV; ++i) {
            c0[i] = side == 0 ? out[i].x : out[i].y;  // the cell next to the face
            c1[i] = side == 0 ? out[i].y : out[i].x;
          }
          pm::x_face_layers(m, side == 0 ? wt.xlo : wt.xhi, c0, c1, g1, g2);
          const long long at = side == 0 ? L.at(-2, y, z) : L.at(L.nx, y, z);
#pragma unroll
          for (int i = 0; i < NV; ++i)
            *reinterpret_cast<float2*>(fout + i * L.fs + at) =
                side == 0 ? make_float2(g2[i], g1[i]) : make_float2(g1[i], g2[i]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      if (SCHEME == LBM_SCHEME_UPWIND2) h2[i] = h1[i];
      h1[i] = F[i];
      F[i] = Z1[i];
    }
    // ring plane k+3 (needed next step) must have landed; the barrier also
    // marks plane k as retired, so its slot takes plane k + NSLOT
    const bool ok = (k + 3 < nplanes) ? arrived(k + 3) : true;
    if (G::SPLIT) {
      // this half is done with plane k; the second half to say so refills its slot
      const unsigned hf = (unsigned)tid >> 7;
      if (half_sync_or(1u + hf, !ok)) {
        timed_out = true;
        break;
      }
      if ((tid & 127) == 0) {
        __threadfence_block();
        const unsigned prev = atomicAdd(&rel[(jb + (unsigned)k) % NSLOT], 1u);
        if ((prev & 1u) && k + NSLOT < nplanes) {
          __threadfence_block();
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue(k + NSLOT);
        }
      }
    } else {
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
      if (tid == 0 && k + NSLOT < nplanes) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(k + NSLOT);
      }
    }
  }
  // SPLIT halves leave the loop on their own (a half that timed out stops
  // releasing slots, so the other one's waits run out too): rejoin here
  if (G::SPLIT) timed_out = __syncthreads_or(timed_out) != 0;

  if (nzc > 0 && !timed_out) {
    const float mr[2] = {hmin_rho.x, hmin_rho.y}, mt[2] = {hmin_T.x, hmin_T.y}, hs[2] = {hsum.x, hsum.y};
    const bool on[2] = {act0, act1};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!on[h]) continue;
      if (!(mr[h] > 0.f)) bad |= LBM_HEALTH_RHO;
      if (!(mt[h] > 0.f)) bad |= LBM_HEALTH_T;
      if (!(fabsf(hs[h]) < 1e30f)) bad |= LBM_HEALTH_NONFINITE;
    }
  }
  if (tid == 0 && timed_out) atomicOr(flags, (unsigned)LBM_HEALTH_TIMEOUT);
  if (bad) atomicOr(flags, bad);
  if (timed_out) {
    // leave no copy in flight: the newest plane of each slot is waited for (bounded)
    if (tid == 0) {
      const int n_issued = G::SPLIT ? *issued_s : issued;
      for (int j = max(0, n_issued - NSLOT); j < n_issued; ++j) drained(j);
    }
    __syncthreads();
  }
  jb += (unsigned)nplanes;
}

// FULL: full tiles; R1: dt = tau (dt/tau = 1, keep_2 = 0), used with FULL only
template <int SCHEME, bool WT, class G, bool FULL, bool R1 = false>
__global__ void __launch_bounds__(G::THREADS, G::CTAS_PER_SM)
    step_pair_kernel(const __grid_constant__ CUtensorMap tin, const float* __restrict__ fin, float* __restrict__ fout,
                     Layout L, Model<float> m, WtDesc wt, RecoverDesc rd, ZSched zs, unsigned* __restrict__ flags,
                     unsigned wait_limit) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::NSLOT * G::SLOT_STRIDE);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < G::NSLOT; ++s) mbar_init(&bars[s], 1);
    if (G::SPLIT) {
      unsigned* rel = reinterpret_cast<unsigned*>(bars + G::NSLOT);
      for (int s = 0; s < G::NSLOT; ++s) rel[s] = 0u;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned jb = 0;
  bool timed_out = false;
  pair_unit<SCHEME, WT, G, FULL, R1>(&tin, fin, fout, L, m, wt, rd, blockIdx.x * G::TX, blockIdx.y * G::TY,
                           zs.z0(blockIdx.z), zs.len(blockIdx.z, L.nz), flags, smem, bars, jb, timed_out, wait_limit);
}

// Persistent batched step: two CTAs per SM take the units of every grid in
// the descriptor table (grid-major, then z chunk, then tile; each unit one
// z-march of a TX x TY column of one grid) from a work queue, one atomic
// increment per unit, so fast and slow CTAs balance.  Every CTA overshoots
// the queue once; the last CTA to finish resets the queue for the next
// launch (stream order), which keeps the launch replayable in a CUDA graph.
// FULL / R1: every grid of the table has full tiles / dt = tau (NND only).
template <int SCHEME, class G, bool FULL = false, bool R1 = false>
__global__ void __launch_bounds__(G::THREADS, G::CTAS_PER_SM)
    step_pair_batch_kernel(const __grid_constant__ BatchTable tab) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::NSLOT * G::SLOT_STRIDE);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < G::NSLOT; ++s) mbar_init(&bars[s], 1);
    if (G::SPLIT) {
      unsigned* rel = reinterpret_cast<unsigned*>(bars + G::NSLOT);
      for (int s = 0; s < G::NSLOT; ++s) rel[s] = 0u;
    }
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
    // the unit's descriptors as locals: read through the runtime index e, the
    // table's constants would otherwise be re-loaded at every use in the plane
    // loop (256^3 alone: 0.497 -> 0.469 ms; eight 128^3: 0.556 -> 0.525 ms)
    const Layout L = it.L;
    const Model<float> m = it.m;
    const WtDesc wt = it.wt;
    const RecoverDesc rd = it.rd;
    const ZSched zs = it.zs;
    pair_unit<SCHEME, true, G, FULL, R1>(&tab.map[e], it.fin, it.fout, L, m, wt, rd, (t % it.tiles_x) * G::TX,
                                         (t / it.tiles_x) * G::TY, zs.z0(chunk), zs.len(chunk, L.nz), it.flags, smem,
                                         bars, jb, timed_out, tab.wait_limit);
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

template <int SCHEME, class G>
cudaError_t set_attributes() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* fn) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  };
  set((const void*)step_pair_kernel<SCHEME, true, G, false>);
  set((const void*)step_pair_kernel<SCHEME, false, G, false>);
  if (SCHEME == LBM_SCHEME_NND) {
    set((const void*)step_pair_kernel<SCHEME, true, G, true>);
    set((const void*)step_pair_kernel<SCHEME, false, G, true>);
    set((const void*)step_pair_kernel<SCHEME, true, G, true, true>);
    set((const void*)step_pair_kernel<SCHEME, false, G, true, true>);
  }
  set((const void*)step_pair_batch_kernel<SCHEME, G>);
  if (SCHEME == LBM_SCHEME_NND) {
    set((const void*)step_pair_batch_kernel<SCHEME, G, true>);
    set((const void*)step_pair_batch_kernel<SCHEME, G, true, true>);
  }
  return e;
}

// The full-tile form (NND only): grids whose nx and ny are multiples of the tile.
template <int SCHEME, bool WT, class G>
void launch_full_or_not(dim3 grid, const CUtensorMap& map, const float* fin, float* fout, const Layout& L,
                        const Model<float>& m, const WtDesc& wt, const RecoverDesc& rd, const ZSched& zs,
                        unsigned* flags, unsigned wait_limit, cudaStream_t st) {
  constexpr bool NND = SCHEME == LBM_SCHEME_NND;
  if (NND && L.nx % G::TX == 0 && L.ny % G::TY == 0 && m.dt_tau == 1.0f && m.keep2 == 0.0f)
    step_pair_kernel<SCHEME, WT, G, NND, NND><<<grid, G::THREADS, G::SMEM, st>>>(map, fin, fout, L, m, wt, rd, zs,
                                                                                  flags, wait_limit);
  else if (NND && L.nx % G::TX == 0 && L.ny % G::TY == 0)
    step_pair_kernel<SCHEME, WT, G, NND><<<grid, G::THREADS, G::SMEM, st>>>(map, fin, fout, L, m, wt, rd, zs, flags,
                                                                             wait_limit);
  else
    step_pair_kernel<SCHEME, WT, G, false><<<grid, G::THREADS, G::SMEM, st>>>(map, fin, fout, L, m, wt, rd, zs,
                                                                               flags, wait_limit);
}

template <int SCHEME, class G>
cudaError_t launch_scheme(const CUtensorMap& map, const float* fin, float* fout, const Layout& L,
                          const Model<float>& m, const WtDesc& wt, const RecoverDesc& rd, const ZSched& zs,
                          unsigned* flags, unsigned wait_limit, cudaStream_t st) {
  dim3 grid((L.nx + G::TX - 1) / G::TX, (L.ny + G::TY - 1) / G::TY, zs.nch);
  const bool any = wt.per[0] || wt.per[1] || wt.per[2] || wt.xlo || wt.xhi;
  if (any)
    launch_full_or_not<SCHEME, true, G>(grid, map, fin, fout, L, m, wt, rd, zs, flags, wait_limit, st);
  else
    launch_full_or_not<SCHEME, false, G>(grid, map, fin, fout, L, m, wt, rd, zs, flags, wait_limit, st);
  return cudaGetLastError();
}

template <class G>
cudaError_t launch_geo(int scheme, const CUtensorMap& map, const float* fin, float* fout, const Layout& L,
                       const Model<float>& m, const WtDesc& wt, const RecoverDesc& rd, const ZSched& zs,
                       unsigned* flags, unsigned wait_limit, cudaStream_t st) {
  switch (scheme) {
    case LBM_SCHEME_NND:
      return launch_scheme<LBM_SCHEME_NND, G>(map, fin, fout, L, m, wt, rd, zs, flags, wait_limit, st);
    case LBM_SCHEME_UPWIND2:
      return launch_scheme<LBM_SCHEME_UPWIND2, G>(map, fin, fout, L, m, wt, rd, zs, flags, wait_limit, st);
    default: return launch_scheme<LBM_SCHEME_UPWIND1, G>(map, fin, fout, L, m, wt, rd, zs, flags, wait_limit, st);
  }
}

template <class G>
cudaError_t prepare_geo() {
  cudaError_t e = set_attributes<LBM_SCHEME_NND, G>();
  if (e == cudaSuccess) e = set_attributes<LBM_SCHEME_UPWIND2, G>();
  if (e == cudaSuccess) e = set_attributes<LBM_SCHEME_UPWIND1, G>();
  return e;
}

}  // namespace

cudaError_t prepare_pair_kernels() {
  cudaError_t e = prepare_geo<Geo64>();
  if (e == cudaSuccess) e = prepare_geo<Geo32>();
  return e;
}

PairShape pair_shape(int cols) {
  if (cols == 64) return {Geo64::TX, Geo64::TY, Geo64::BX, Geo64::BY, Geo64::THREADS, Geo64::CTAS_PER_SM};
  return {Geo32::TX, Geo32::TY, Geo32::BX, Geo32::BY, Geo32::THREADS, Geo32::CTAS_PER_SM};
}

template <class G>
void launch_batch_geo(int scheme, const BatchTable& tab, int grid, cudaStream_t st) {
  // the full-tile and dt = tau forms when every grid of the table qualifies
  bool full = true, r1 = true;
  for (int e = 0; e < tab.n; ++e) {
    const BatchItem& it = tab.item[e];
    full = full && it.L.nx % G::TX == 0 && it.L.ny % G::TY == 0;
    r1 = r1 && it.m.dt_tau == 1.0f && it.m.keep2 == 0.0f;
  }
  switch (scheme) {
    case LBM_SCHEME_NND:
      if (full && r1) step_pair_batch_kernel<LBM_SCHEME_NND, G, true, true><<<grid, G::THREADS, G::SMEM, st>>>(tab);
      else if (full) step_pair_batch_kernel<LBM_SCHEME_NND, G, true><<<grid, G::THREADS, G::SMEM, st>>>(tab);
      else step_pair_batch_kernel<LBM_SCHEME_NND, G><<<grid, G::THREADS, G::SMEM, st>>>(tab);
      break;
    case LBM_SCHEME_UPWIND2:
      step_pair_batch_kernel<LBM_SCHEME_UPWIND2, G><<<grid, G::THREADS, G::SMEM, st>>>(tab);
      break;
    default: step_pair_batch_kernel<LBM_SCHEME_UPWIND1, G><<<grid, G::THREADS, G::SMEM, st>>>(tab);
  }
}

cudaError_t launch_step_pair_batch(int cols, int scheme, const BatchTable& tab, int grid, cudaStream_t st) {
  if (cols == 64) launch_batch_geo<Geo64>(scheme, tab, grid, st);
  else launch_batch_geo<Geo32>(scheme, tab, grid, st);
  return cudaGetLastError();
}

cudaError_t launch_step_pair(int cols, int scheme, const CUtensorMap& map, const float* fin, float* fout,
                             const Layout& L, const Model<float>& m, const WtDesc& wt, const RecoverDesc& rd,
                             const ZSched& zs, unsigned* flags, unsigned wait_limit, cudaStream_t st) {
  if (cols == 64) return launch_geo<Geo64>(scheme, map, fin, fout, L, m, wt, rd, zs, flags, wait_limit, st);
  return launch_geo<Geo32>(scheme, map, fin, fout, L, m, wt, rd, zs, flags, wait_limit, st);
}

// 1/x as the FP32 step kernels form the inverse density (pm::rcp2), two
// values per thread; an odd tail pads its second lane with 1.
__global__ void __launch_bounds__(256) reciprocal_kernel(const float* __restrict__ x, float* __restrict__ y,
                                                         long long n) {
  const long long stride = 2LL * gridDim.x * blockDim.x;
  for (long long i = 2LL * ((long long)blockIdx.x * blockDim.x + threadIdx.x); i < n; i += stride) {
    const bool two = i + 1 < n;
    const float2 r = pm::rcp2(make_float2(x[i], two ? x[i + 1] : 1.f));
    y[i] = r.x;
    if (two) y[i + 1] = r.y;
  }
}

cudaError_t launch_reciprocal_fp32(const float* x, float* y, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long pairs = (n + 1) / 2;
  const int blocks = (int)std::min<long long>((pairs + 255) / 256, 152LL * 8);
  reciprocal_kernel<<<blocks, 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}

}  // namespace lbm
