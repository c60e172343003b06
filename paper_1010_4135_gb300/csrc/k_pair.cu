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
// without the prefetch).
using Geo32 = PairGeo<ring::TX, ring::TY, 2>;
// 64 x 8 tiles (box 72 x 12 x 1 x 15): one CTA of 8 warps per SM, 288-byte
// row reads, run as two split halves.  Its data movement alone (ring +
// stores, no arithmetic) is faster (0.362 ms against 0.443 ms on 256^3);
// with the arithmetic it takes 0.511 ms (0.549 ms with one CTA-wide barrier
// per plane), against 0.465 ms for two independent 32 x 8 CTAs per SM.
using Geo64 = PairGeo<64, 8, 2, true>;
static_assert(Geo32::BX == ring::BX && Geo32::BY == ring::BY, "Geo32 shares the tiled kernel's tensor map");

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// minmod(x, d) given lo = min(d, 0), hi = max(d, 0): exact.
__device__ __forceinline__ float mmc(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }
__device__ __forceinline__ float2 mmc2(float2 x, float2 d) {
  return make_float2(mmc(x.x, fminf(d.x, 0.f), fmaxf(d.x, 0.f)), mmc(x.y, fminf(d.y, 0.f), fmaxf(d.y, 0.f)));
}

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

__device__ __forceinline__ int wrapi(int k, int n) {
  const int r = k % n;
  return r < 0 ? r + n : r;
}

// rho, u, T of one cell from its 15 values (stride pl floats) in FP64
// (relations e1-e3 summed in double); out of line, called only for cells
// whose FP32 recovery is ill-conditioned (RecoverDesc).
struct Macro1 {
  float rho, ux, uy, uz, T;
};
__device__ __noinline__ Macro1 recover_fp64(const float* q, int pl, double c1, double s, double eta0sq,
                                            double c1sq, double c2sq, double inv_b) {
  double f[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) f[i] = (double)q[i * pl];
  const double sa = ((f[1] + f[2]) + (f[3] + f[4])) + (f[5] + f[6]);
  const double dpp = f[7] + f[8], dpm = f[9] + f[10], dmp = f[11] + f[12], dmm = f[13] + f[14];
  const double sd = (dpp + dpm) + (dmp + dmm);
  const double rho = f[0] + sa + sd;
  const double mx = c1 * (f[1] - f[2]) + s * ((dpp + dpm) - (dmp + dmm));
  const double my = c1 * (f[3] - f[4]) + s * ((dpp + dmp) - (dpm + dmm));
  const double mz = c1 * (f[5] - f[6]) + s * (((f[7] + f[9]) + (f[11] + f[13])) - ((f[8] + f[10]) + (f[12] + f[14])));
  const double E = eta0sq * f[0] + c1sq * sa + c2sq * sd;
  const double ux = mx / rho, uy = my / rho, uz = mz / rho;
  const double T = (E / rho - (ux * ux + uy * uy + uz * uz)) * inv_b;
  return {(float)rho, (float)ux, (float)uy, (float)uz, (float)T};
}

// The two layers outside an x face from the boundary cell c0 (next to the
// face) and its neighbour c1 (Sec. 4(2)): g1 next to the face, g2 outside it.
__device__ __forceinline__ void x_face_layers(const Model<float>& m, int kind, const float c0[NV], const float c1[NV],
                                              float g1[NV], float g2[NV]) {
  float M0[5], M1[5], G1[5], G2[5];
  moments(m, c0, M0[0], M0[1], M0[2], M0[3], M0[4]);
  if (kind == LBM_BC_EXTRAPOLATE) {
    moments(m, c1, M1[0], M1[1], M1[2], M1[3], M1[4]);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      G1[q] = 2.f * M0[q] - M1[q];
      G2[q] = 2.f * G1[q] - M0[q];
    }
  } else {  // LBM_BC_REFLECT, normal velocity u1
#pragma unroll
    for (int q = 0; q < 5; ++q) G1[q] = G2[q] = M0[q];
    G1[1] = 0.f;
    G2[1] = -M0[1];
  }
  equilibrium(m, G1[0], G1[1], G1[2], G1[3], G1[4], g1);
  equilibrium(m, G2[0], G2[1], G2[2], G2[3], G2[4], g2);
}

// One z-march unit: the TX x TY column at (x0, y0), planes z0 .. z0+nzc-1.
// Plane j of the unit is the ring's plane number jb + j (slot (jb+j) % NSLOT,
// phase parity ((jb+j) / NSLOT) & 1), so consecutive units of a CTA keep
// using the same barriers; jb advances by the unit's plane count.  All
// threads of the CTA call it together; timed_out is uniform.
template <int SCHEME, bool WT, class G>
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
  const bool act0 = (x < L.nx) && (y < L.ny);
  const bool act1 = (x + 1 < L.nx) && (y < L.ny);
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
    for (int i = 0; i < NV; ++i) {
      const int sz = vsign(i, 2);
      const float2 fc = ld2(P0 + i * PL + c);
      if (sz > 0) carry[i] = mmc2(sub(h1[i], h2[i]), sub(fc, h1[i]));
      if (sz < 0) carry[i] = mmc2(sub(ld2(P1 + i * PL + c), fc), sub(fc, h1[i]));
    }
  }

  const float2 half = bc2(0.5f);
  // F: the own pair of cell plane k; Fn: that of plane k+1, read as the z
  // neighbour during plane k and kept in registers for the next plane
  float2 F[NV], Fn[NV];
  if (!timed_out) {
    const float* Q0 = slot(0);
#pragma unroll
    for (int i = 0; i < NV; ++i) F[i] = ld2(Q0 + i * PL + c);
  }
  for (int k = 0; k < nzc && !timed_out; ++k) {
    const float* P0 = slot(k);
    const float* P1 = slot(k + 1);
    const float* P2 = slot(k + 2);


    // moments (relations e1-e3)
    const float2 sa = add(add(add(F[1], F[2]), add(F[3], F[4])), add(F[5], F[6]));
    const float2 dpp = add(F[7], F[8]), dpm = add(F[9], F[10]), dmp = add(F[11], F[12]), dmm = add(F[13], F[14]);
    const float2 sd = add(add(dpp, dpm), add(dmp, dmm));
    float2 rho = add(add(F[0], sa), sd);
    const float2 mx = fma2(bc2(m.c1), sub(F[1], F[2]), mul(bc2(m.s), sub(add(dpp, dpm), add(dmp, dmm))));
    const float2 my = fma2(bc2(m.c1), sub(F[3], F[4]), mul(bc2(m.s), sub(add(dpp, dmp), add(dpm, dmm))));
    const float2 mz = fma2(bc2(m.c1), sub(F[5], F[6]),
                           mul(bc2(m.s), sub(add(add(F[7], F[9]), add(F[11], F[13])),
                                             add(add(F[8], F[10]), add(F[12], F[14])))));
    const float2 E = fma2(bc2(m.eta0sq), F[0], fma2(bc2(m.c1sq), sa, mul(bc2(m.c2sq), sd)));
    const float2 ir = make_float2(__frcp_rn(rho.x), __frcp_rn(rho.y));
    float2 ux = mul(mx, ir), uy = mul(my, ir), uz = mul(mz, ir);
    float2 usq = fma2(ux, ux, fma2(uy, uy, mul(uz, uz)));
    float2 T = mul(sub(mul(E, ir), usq), bc2(m.inv_b));
    if (rd.on) {
      // ill-conditioned FP32 temperature (RecoverDesc): redo the cell in FP64
      const float2 Aa = fma2(bc2(m.AaT), T, fma2(bc2(m.AaU), usq, bc2(m.Aa0)));
      const float2 Ad = fma2(bc2(m.AdT), T, fma2(bc2(m.AdU), usq, bc2(m.Ad0)));
      const float lhs0 = fmaf(rd.axis_w, fabsf(Aa.x), fmaf(rd.diag_w, fabsf(Ad.x), usq.x));
      const float lhs1 = fmaf(rd.axis_w, fabsf(Aa.y), fmaf(rd.diag_w, fabsf(Ad.y), usq.y));
      const bool need0 = act0 && !(lhs0 <= rd.thresh_b * T.x);
      const bool need1 = act1 && !(lhs1 <= rd.thresh_b * T.y);
      if (need0 || need1) {
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          if (!(h == 0 ? need0 : need1)) continue;
          const Macro1 r = recover_fp64(P0 + c + h, PL, rd.c1, rd.s, rd.eta0sq, rd.c1sq, rd.c2sq, rd.inv_b);
          if (h == 0) {
            rho.x = r.rho; ux.x = r.ux; uy.x = r.uy; uz.x = r.uz; T.x = r.T;
          } else {
            rho.y = r.rho; ux.y = r.ux; uy.y = r.uy; uz.y = r.uz; T.y = r.T;
          }
        }
        usq = fma2(ux, ux, fma2(uy, uy, mul(uz, uz)));
      }
    }
    {
      const float ax[2] = {rho.x, rho.y}, tt[2] = {T.x, T.y};
      const float chk[2] = {fabsf(rho.x) + fabsf(T.x) + fabsf(ux.x) + fabsf(uy.x) + fabsf(uz.x),
                            fabsf(rho.y) + fabsf(T.y) + fabsf(ux.y) + fabsf(uy.y) + fabsf(uz.y)};
      const bool on[2] = {act0, act1};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!on[h]) continue;
        if (!(ax[h] > 0.f)) bad |= LBM_HEALTH_RHO;
        if (!(tt[h] > 0.f)) bad |= LBM_HEALTH_T;
        if (!(chk[h] < 1e30f)) bad |= LBM_HEALTH_NONFINITE;
      }
    }
    // equilibrium (Eq. "eq"), per shell A + B w + D w^2
    float2 feq[NV];
    feq[0] = mul(rho, mul(bc2(m.AR), T));
    {
      const float2 Aa = fma2(bc2(m.AaT), T, fma2(bc2(m.AaU), usq, bc2(m.Aa0)));
      const float2 Ba = fma2(bc2(m.BaT), T, fma2(bc2(m.BaU), usq, bc2(m.Ba0)));
      const float2 u3[3] = {ux, uy, uz};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float2 w = mul(bc2(m.c1), u3[a]);
        const float2 q = fma2(bc2(m.Da), mul(w, w), Aa);
        const float2 l = mul(Ba, w);
        feq[1 + 2 * a] = mul(rho, add(q, l));
        feq[2 + 2 * a] = mul(rho, sub(q, l));
      }
      const float2 Ad = fma2(bc2(m.AdT), T, fma2(bc2(m.AdU), usq, bc2(m.Ad0)));
      const float2 Bd = fma2(bc2(m.BdT), T, fma2(bc2(m.BdU), usq, bc2(m.Bd0)));
      const float2 sxy = add(ux, uy), dxy = sub(ux, uy);
      const float2 w4[4] = {mul(bc2(m.s), add(sxy, uz)), mul(bc2(m.s), sub(sxy, uz)), mul(bc2(m.s), add(dxy, uz)),
                            mul(bc2(m.s), sub(dxy, uz))};
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float2 q = fma2(bc2(m.Dd), mul(w4[kk], w4[kk]), Ad);
        const float2 l = mul(Bd, w4[kk]);
        feq[7 + kk] = mul(rho, add(q, l));
        feq[14 - kk] = mul(rho, sub(q, l));
      }
    }

    float2 out[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float* q = P0 + i * PL + c;
      const float2 B = F[i];
      float2 conv = make_float2(0.f, 0.f);
      float2 S = make_float2(0.f, 0.f);
      // ---- x: neighbour pairs A = (x-2, x-1), C = (x+2, x+3)
      {
        const int sg = vsign(i, 0);
        if (sg != 0 || i <= 6) {
          const float2 A = ld2(q - 2), C = ld2(q + 2);
          const float e1 = B.x - A.y, e2 = B.y - B.x, e3 = C.x - B.y;
          if (sg > 0) {
            const float e0 = A.y - A.x;
            float2 G;
            if (SCHEME == LBM_SCHEME_NND) {
              const float lo1 = fminf(e1, 0.f), hi1 = fmaxf(e1, 0.f);
              const float m12 = mmc(e2, lo1, hi1), m01 = mmc(e0, lo1, hi1);
              const float m23 = mmc(e3, fminf(e2, 0.f), fmaxf(e2, 0.f));
              G = fma2(half, sub(make_float2(m12, m23), make_float2(m01, m12)), make_float2(e1, e2));
            } else if (SCHEME == LBM_SCHEME_UPWIND2) {
              // (3 c - 4 m1 + m2) / 2: cell x (A.x, A.y, B.x), cell x+1 (A.y, B.x, B.y)
              G = mul(half, add(fma2(bc2(3.f), B, mul(bc2(-4.f), make_float2(A.y, B.x))), A));
            } else {
              G = make_float2(e1, e2);
            }
            conv = add(conv, G);
          } else if (sg < 0) {
            const float e4 = C.y - C.x;
            float2 G;
            if (SCHEME == LBM_SCHEME_NND) {
              const float lo2 = fminf(e2, 0.f), hi2 = fmaxf(e2, 0.f);
              const float m23 = mmc(e3, lo2, hi2), m12 = mmc(e1, lo2, hi2);
              const float m34 = mmc(e4, fminf(e3, 0.f), fmaxf(e3, 0.f));
              G = fma2(bc2(-0.5f), sub(make_float2(m23, m34), make_float2(m12, m23)), make_float2(e2, e3));
            } else if (SCHEME == LBM_SCHEME_UPWIND2) {
              // (4 p1 - 3 c - p2) / 2: cell x (B.x, B.y, C.x), cell x+1 (B.y, C.x, C.y)
              const float2 P1x = make_float2(B.y, C.x);
              G = mul(half, sub(fma2(bc2(4.f), P1x, mul(bc2(-3.f), B)), C));
            } else {
              G = make_float2(e2, e3);
            }
            conv = sub(conv, G);
          }
          if (i <= 6) S = add(S, make_float2(A.y + B.y, B.x + C.x));
        }
      }
      // ---- y: rows y-2 .. y+2 of the same pair
      {
        const int sg = vsign(i, 1);
        if (sg != 0 || i <= 6) {
          const float2 M1 = ld2(q - BX), P1y = ld2(q + BX);
          if (sg > 0) {
            const float2 M2 = ld2(q - 2 * BX);
            const float2 D0 = sub(B, M1);
            float2 G;
            if (SCHEME == LBM_SCHEME_NND) {
              G = fma2(half, sub(mmc2(sub(P1y, B), D0), mmc2(sub(M1, M2), D0)), D0);
            } else if (SCHEME == LBM_SCHEME_UPWIND2) {
              G = mul(half, add(fma2(bc2(3.f), B, mul(bc2(-4.f), M1)), M2));
            } else {
              G = D0;
            }
            conv = add(conv, G);
          } else if (sg < 0) {
            const float2 P2y = ld2(q + 2 * BX);
            const float2 D1 = sub(P1y, B);
            float2 G;
            if (SCHEME == LBM_SCHEME_NND) {
              G = fma2(bc2(-0.5f), sub(mmc2(sub(P2y, P1y), D1), mmc2(sub(B, M1), D1)), D1);
            } else if (SCHEME == LBM_SCHEME_UPWIND2) {
              G = mul(half, sub(fma2(bc2(4.f), P1y, mul(bc2(-3.f), B)), P2y));
            } else {
              G = D1;
            }
            conv = sub(conv, G);
          }
          if (i <= 6) S = add(S, add(M1, P1y));
        }
      }
      // ---- z: planes z+1, z+2 from the ring, z-1 (z-2) from registers
      {
        const int sg = vsign(i, 2);
        const float2 Z1 = ld2(P1 + i * PL + c);
        Fn[i] = Z1;
        const float2 H = h1[i];
        if (sg > 0) {
          const float2 D0 = sub(B, H);
          float2 G;
          if (SCHEME == LBM_SCHEME_NND) {
            const float2 mA = mmc2(sub(Z1, B), D0);
            G = fma2(half, sub(mA, carry[i]), D0);
            carry[i] = mA;
          } else if (SCHEME == LBM_SCHEME_UPWIND2) {
            G = mul(half, add(fma2(bc2(3.f), B, mul(bc2(-4.f), H)), h2[i]));
          } else {
            G = D0;
          }
          conv = add(conv, G);
        } else if (sg < 0) {
          const float2 Z2 = ld2(P2 + i * PL + c);
          const float2 D1 = sub(Z1, B);
          float2 G;
          if (SCHEME == LBM_SCHEME_NND) {
            const float2 mA = mmc2(sub(Z2, Z1), D1);
            G = fma2(bc2(-0.5f), sub(mA, carry[i]), D1);
            carry[i] = mA;
          } else if (SCHEME == LBM_SCHEME_UPWIND2) {
            G = mul(half, sub(fma2(bc2(4.f), Z1, mul(bc2(-3.f), B)), Z2));
          } else {
            G = D1;
          }
          conv = sub(conv, G);
        }
        if (i <= 6) S = add(S, add(H, Z1));
      }
      const float keep = i == 0 ? m.keep0 : (i <= 6 ? m.keep1 : m.keep2);
      const float kk = i == 0 ? 0.f : (i <= 6 ? m.k1 : m.k2);
      const float lam = i == 0 ? m.lam0 : (i <= 6 ? m.lam1 : 0.f);
      float2 o = fma2(bc2(m.dt_tau), feq[i], mul(bc2(keep), B));
      if (i != 0) o = fma2(bc2(-kk), conv, o);
      if (i <= 6) o = fma2(bc2(lam), S, o);
      out[i] = o;
    }
    const long long g = gbase + (long long)k * L.plane;
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
            for (int i = 0; i < NV; ++i) *reinterpret_cast<float2*>(fout + i * L.fs + at) = out[i];
          } else {
#pragma unroll
            for (int i = 0; i < NV; ++i) fout[i * L.fs + at] = out[i].x;
          }
        }
      }
      const bool lo = wt.xlo && x == 0, hi = wt.xhi && x == L.nx - 2;
      if (lo || hi) {
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
          if (side == 0 ? !lo : !hi) continue;
          float c0[NV], c1[NV], g1[NV], g2[NV];
#pragma unroll
          for (int i = 0; i < NV; ++i) {
            c0[i] = side == 0 ? out[i].x : out[i].y;  // the cell next to the face
            c1[i] = side == 0 ? out[i].y : out[i].x;
          }
          x_face_layers(m, side == 0 ? wt.xlo : wt.xhi, c0, c1, g1, g2);
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
      h2[i] = h1[i];
      h1[i] = F[i];
      F[i] = Fn[i];
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

template <int SCHEME, bool WT, class G>
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
  pair_unit<SCHEME, WT, G>(&tin, fin, fout, L, m, wt, rd, blockIdx.x * G::TX, blockIdx.y * G::TY,
                           zs.z0(blockIdx.z), zs.len(blockIdx.z, L.nz), flags, smem, bars, jb, timed_out, wait_limit);
}

// Persistent batched step: two CTAs per SM take the units of every grid in
// the descriptor table (grid-major, then z chunk, then tile; each unit one
// z-march of a TX x TY column of one grid) from a work queue, one atomic
// increment per unit, so fast and slow CTAs balance.  Every CTA overshoots
// the queue once; the last CTA to finish resets the queue for the next
// launch (stream order), which keeps the launch replayable in a CUDA graph.
template <int SCHEME, class G>
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
    pair_unit<SCHEME, true, G>(&tab.map[e], it.fin, it.fout, L, m, wt, rd, (t % it.tiles_x) * G::TX,
                               (t / it.tiles_x) * G::TY, zs.z0(chunk), zs.len(chunk, L.nz), it.flags, smem, bars,
                               jb, timed_out, tab.wait_limit);
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
  cudaError_t e = cudaFuncSetAttribute(step_pair_kernel<SCHEME, true, G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_pair_kernel<SCHEME, false, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_pair_batch_kernel<SCHEME, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G::SMEM);
  return e;
}

template <int SCHEME, class G>
cudaError_t launch_scheme(const CUtensorMap& map, const float* fin, float* fout, const Layout& L,
                          const Model<float>& m, const WtDesc& wt, const RecoverDesc& rd, const ZSched& zs,
                          unsigned* flags, unsigned wait_limit, cudaStream_t st) {
  dim3 grid((L.nx + G::TX - 1) / G::TX, (L.ny + G::TY - 1) / G::TY, zs.nch);
  const bool any = wt.per[0] || wt.per[1] || wt.per[2] || wt.xlo || wt.xhi;
  if (any)
    step_pair_kernel<SCHEME, true, G><<<grid, G::THREADS, G::SMEM, st>>>(map, fin, fout, L, m, wt, rd, zs, flags,
                                                                         wait_limit);
  else
    step_pair_kernel<SCHEME, false, G><<<grid, G::THREADS, G::SMEM, st>>>(map, fin, fout, L, m, wt, rd, zs, flags,
                                                                          wait_limit);
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
  switch (scheme) {
    case LBM_SCHEME_NND: step_pair_batch_kernel<LBM_SCHEME_NND, G><<<grid, G::THREADS, G::SMEM, st>>>(tab); break;
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

}  // namespace lbm
