// Per-cell-pair arithmetic of the FP32 tiled step kernels (sm_103a).
//
// A thread owns the two x-adjacent cells (x, x+1) of one tile row and holds
// their values as float2; everything that is the same arithmetic for both
// cells runs as packed f32x2 operations (FADD2, FMUL2, FFMA2).  The pair
// kernel (all 15 fields per thread) and the field-split kernel (two warp
// groups of one tile, each updating part of the 15 fields) both inline these
// functions, so they round identically and give bitwise equal results.
//
// Shared-memory plane tiles: field i of a plane tile starts PL floats after
// field i-1; rows are BX floats; `c` indexes the thread's own pair (even).
#pragma once

#include "lbm_internal.cuh"

namespace lbm {
namespace pm {

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return fma2(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// minmod(x, d) given lo = min(d, 0), hi = max(d, 0): exact.
__device__ __forceinline__ float mmc(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }
__device__ __forceinline__ float2 mmc2(float2 x, float2 d) {
  return make_float2(mmc(x.x, fminf(d.x, 0.f), fmaxf(d.x, 0.f)), mmc(x.y, fminf(d.y, 0.f), fmaxf(d.y, 0.f)));
}

// 1/a for both cells: the hardware approximation r0 (PTX rcp.approx.ftz.f32,
// relative error d of a few 2^-23 at most) refined by one Newton-Raphson
// step for the reciprocal, r = r0 - r0 (a r0 - 1) (the iteration
// x <- x (2 - a x) of Newton-Raphson division, written with the residual
// formed by one fma).  With r0 = (1 + d)/a the residual a r0 - 1 = d is exact
// in the fma, and r = (1 - d^2)/a up to the final rounding: |r a - 1| <=
// 2^-24 + d^2 + O(2^-46) while the correction r0 (a r0 - 1) stays normal
// (|a| <= 2^100): the accuracy of one rounding, though not always the nearest
// float.  a = 0 or +-inf (and subnormal a, flushed to 0) give NaN; a
// cell with such a density fails the health checks.  Four packed operations
// and two MUFU against two correctly rounded reciprocals.
__device__ __forceinline__ float2 rcp2(float2 a) {
  float2 r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0.x) : "f"(a.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0.y) : "f"(a.y));
  const float2 res = fma2(a, r0, bc2(-1.f));
  return sub(r0, mul(res, r0));
}

// Macroscopic state of a pair.
struct Mom {
  float2 rho, ux, uy, uz, T, usq;
};

// rho, u, T of one cell from its 15 values (stride pl floats) in FP64
// (relations e1-e3 summed in double); out of line, called only for cells
// whose FP32 recovery is ill-conditioned (RecoverDesc).
struct Macro1 {
  float rho, ux, uy, uz, T;
};
__device__ __noinline__ inline Macro1 recover_fp64(const float* q, int pl, double c1, double s, double eta0sq,
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

// Moments of the pair (relations e1-e3) from its 15 values F; with rd.on,
// cells whose FP32 temperature is ill-conditioned are redone in FP64 from the
// plane tile at P0 + c (field stride PL).
__device__ __forceinline__ Mom moments(const Model<float>& m, const RecoverDesc& rd, const float2 (&F)[NV],
                                       const float* P0, int c, int PL, bool act0, bool act1) {
  const float2 sa = add(add(add(F[1], F[2]), add(F[3], F[4])), add(F[5], F[6]));
  const float2 dpp = add(F[7], F[8]), dpm = add(F[9], F[10]), dmp = add(F[11], F[12]), dmm = add(F[13], F[14]);
  const float2 sd = add(add(dpp, dpm), add(dmp, dmm));
  Mom r;
  r.rho = add(add(F[0], sa), sd);
  const float2 mx = fma2(bc2(m.c1), sub(F[1], F[2]), mul(bc2(m.s), sub(add(dpp, dpm), add(dmp, dmm))));
  const float2 my = fma2(bc2(m.c1), sub(F[3], F[4]), mul(bc2(m.s), sub(add(dpp, dmp), add(dpm, dmm))));
  const float2 mz = fma2(bc2(m.c1), sub(F[5], F[6]),
                         mul(bc2(m.s), sub(add(add(F[7], F[9]), add(F[11], F[13])),
                                           add(add(F[8], F[10]), add(F[12], F[14])))));
  const float2 E = fma2(bc2(m.eta0sq), F[0], fma2(bc2(m.c1sq), sa, mul(bc2(m.c2sq), sd)));
  const float2 ir = rcp2(r.rho);
  r.ux = mul(mx, ir);
  r.uy = mul(my, ir);
  r.uz = mul(mz, ir);
  r.usq = fma2(r.ux, r.ux, fma2(r.uy, r.uy, mul(r.uz, r.uz)));
  r.T = mul(sub(mul(E, ir), r.usq), bc2(m.inv_b));
  if (rd.on) {
    // ill-conditioned FP32 temperature (RecoverDesc): redo the cell in FP64
    const float2 Aa = fma2(bc2(m.AaT), r.T, fma2(bc2(m.AaU), r.usq, bc2(m.Aa0)));
    const float2 Ad = fma2(bc2(m.AdT), r.T, fma2(bc2(m.AdU), r.usq, bc2(m.Ad0)));
    const float lhs0 = fmaf(rd.axis_w, fabsf(Aa.x), fmaf(rd.diag_w, fabsf(Ad.x), r.usq.x));
    const float lhs1 = fmaf(rd.axis_w, fabsf(Aa.y), fmaf(rd.diag_w, fabsf(Ad.y), r.usq.y));
    const bool need0 = act0 && !(lhs0 <= rd.thresh_b * r.T.x);
    const bool need1 = act1 && !(lhs1 <= rd.thresh_b * r.T.y);
    if (need0 || need1) {
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        if (!(h == 0 ? need0 : need1)) continue;
        const Macro1 q = recover_fp64(P0 + c + h, PL, rd.c1, rd.s, rd.eta0sq, rd.c1sq, rd.c2sq, rd.inv_b);
        if (h == 0) {
          r.rho.x = q.rho; r.ux.x = q.ux; r.uy.x = q.uy; r.uz.x = q.uz; r.T.x = q.T;
        } else {
          r.rho.y = q.rho; r.ux.y = q.ux; r.uy.y = q.uy; r.uz.y = q.uz; r.T.y = q.T;
        }
      }
      r.usq = fma2(r.ux, r.ux, fma2(r.uy, r.uy, mul(r.uz, r.uz)));
    }
  }
  return r;
}

// Health bits of the pair's active cells: rho <= 0, T <= 0, non-finite.
__device__ __forceinline__ unsigned health(const Mom& r, bool act0, bool act1) {
  unsigned bad = 0u;
  const float ax[2] = {r.rho.x, r.rho.y}, tt[2] = {r.T.x, r.T.y};
  const float chk[2] = {fabsf(r.rho.x) + fabsf(r.T.x) + fabsf(r.ux.x) + fabsf(r.uy.x) + fabsf(r.uz.x),
                        fabsf(r.rho.y) + fabsf(r.T.y) + fabsf(r.ux.y) + fabsf(r.uy.y) + fabsf(r.uz.y)};
  const bool on[2] = {act0, act1};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!on[h]) continue;
    if (!(ax[h] > 0.f)) bad |= LBM_HEALTH_RHO;
    if (!(tt[h] > 0.f)) bad |= LBM_HEALTH_T;
    if (!(chk[h] < 1e30f)) bad |= LBM_HEALTH_NONFINITE;
  }
  return bad;
}

// f^eq_i of the pair (Eq. "eq"): rho (A + B w + D w^2) per shell, evaluated
// as (rho A + rho D w^2) + rho B w with rho folded into the shell's three
// coefficients once per pair (Shell below) and the linear term fused: one fma
// each, not a product and a sum (the compiler may fuse a packed product into
// a later sum in one kernel and not in another; written as fmas, every
// kernel rounds them the same way).  i is a compile-time constant after
// unrolling.
struct Shell {
  float2 rA, rB, rD;  // rho A, rho B, rho D
};
__device__ __forceinline__ Shell axis_shell(const Model<float>& m, const Mom& r) {
  const float2 A = fma2(bc2(m.AaT), r.T, fma2(bc2(m.AaU), r.usq, bc2(m.Aa0)));
  const float2 B = fma2(bc2(m.BaT), r.T, fma2(bc2(m.BaU), r.usq, bc2(m.Ba0)));
  return {mul(r.rho, A), mul(r.rho, B), mul(r.rho, bc2(m.Da))};
}
__device__ __forceinline__ Shell diag_shell(const Model<float>& m, const Mom& r) {
  const float2 A = fma2(bc2(m.AdT), r.T, fma2(bc2(m.AdU), r.usq, bc2(m.Ad0)));
  const float2 B = fma2(bc2(m.BdT), r.T, fma2(bc2(m.BdU), r.usq, bc2(m.Bd0)));
  return {mul(r.rho, A), mul(r.rho, B), mul(r.rho, bc2(m.Dd))};
}
__device__ __forceinline__ float2 feq(const Model<float>& m, const Mom& r, int i) {
  if (i == 0) return mul(r.rho, mul(bc2(m.AR), r.T));
  if (i <= 6) {
    const Shell sh = axis_shell(m, r);
    const int a = (i - 1) / 2;
    const float2 w = mul(bc2(m.c1), a == 0 ? r.ux : (a == 1 ? r.uy : r.uz));
    const float2 q = fma2(sh.rD, mul(w, w), sh.rA);
    return fma2((i - 1) % 2 == 0 ? sh.rB : neg(sh.rB), w, q);
  }
  const Shell sh = diag_shell(m, r);
  // k = 0..3 are (+ + +), (+ + -), (+ - +), (+ - -); fields 7+k and 14-k are opposite
  const int k = i <= 10 ? i - 7 : 14 - i;
  const float2 sxy = add(r.ux, r.uy), dxy = sub(r.ux, r.uy);
  const float2 w = mul(bc2(m.s), k == 0 ? add(sxy, r.uz) : (k == 1 ? sub(sxy, r.uz) : (k == 2 ? add(dxy, r.uz) : sub(dxy, r.uz))));
  const float2 q = fma2(sh.rD, mul(w, w), sh.rA);
  return fma2(i <= 10 ? sh.rB : neg(sh.rB), w, q);
}

// New value of field i of the pair (i a compile-time constant after
// unrolling): the NND (or upwind) convection of Sec. 3 along x, y, z, the
// extra dissipation for i <= 6 and the BGK update, with relaxation and the
// Laplacian centre folded into keep_i:
//   f_new = keep_i f + (dt/tau) f^eq - (|v| dt/dx) C + (lambda_i dt/dx^2) S.
// q: the pair in plane tile k (field i); Z1: the pair in plane k+1, Z2p: the
// field's tile in plane k+2 at the pair; h1, h2: the pair in planes k-1, k-2
// (registers); carry: the minmod of the lower z interface (NND), replaced by
// that of the upper one.  DZ (NND, diagonal velocities with v_z > 0): the
// lower z difference f_k - f_{k-1} is carried in dz (the upper difference of
// the plane before, the same rounded value) instead of being formed from H,
// and dz takes this plane's upper difference.
template <int SCHEME, int BX, bool DZ = false, bool R1 = false>
__device__ __forceinline__ float2 field_update(const Model<float>& m, int i, const float* q, float2 B, float2 Z1,
                                               const float* Z2p, float2 H, float2 H2, float2& carry, float2& dz,
                                               float2 fe) {
  const float2 half = bc2(0.5f);
  // the convection and neighbour sums start from their first term (0 + x is
  // not an identity for x = -0, so the compiler keeps an add with 0); conv
  // holds the negated sum when its first term enters with a minus sign (cneg),
  // folded into the coefficient at the end.  i is a compile-time constant, so
  // the bookkeeping folds away.
  float2 conv = make_float2(0.f, 0.f), S = make_float2(0.f, 0.f);
  bool have_c = false, cneg = false, have_s = false;
  auto acc = [&](float2 G, bool plus) {
    if (!have_c) {
      conv = G;
      cneg = !plus;
      have_c = true;
    } else {
      conv = (plus != cneg) ? add(conv, G) : sub(conv, G);
    }
  };
  auto nsum = [&](float2 v) {
    S = have_s ? add(S, v) : v;
    have_s = true;
  };
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
        acc(G, true);
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
        acc(G, false);
      }
      if (i <= 6) nsum(make_float2(A.y + B.y, B.x + C.x));
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
        acc(G, true);
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
        acc(G, false);
      }
      if (i <= 6) nsum(add(M1, P1y));
    }
  }
  // ---- z: planes z+1, z+2 from the ring, z-1 (z-2) from registers
  {
    const int sg = vsign(i, 2);
    if (sg > 0) {
      constexpr bool kCarried = DZ && SCHEME == LBM_SCHEME_NND;
      const float2 D0 = (kCarried && i >= 7) ? dz : sub(B, H);
      float2 G;
      if (SCHEME == LBM_SCHEME_NND) {
        const float2 Dup = sub(Z1, B);
        const float2 mA = mmc2(Dup, D0);
        G = fma2(half, sub(mA, carry), D0);
        carry = mA;
        if (kCarried && i >= 7) dz = Dup;
      } else if (SCHEME == LBM_SCHEME_UPWIND2) {
        G = mul(half, add(fma2(bc2(3.f), B, mul(bc2(-4.f), H)), H2));
      } else {
        G = D0;
      }
      acc(G, true);
    } else if (sg < 0) {
      const float2 Z2 = ld2(Z2p);
      const float2 D1 = sub(Z1, B);
      float2 G;
      if (SCHEME == LBM_SCHEME_NND) {
        const float2 mA = mmc2(sub(Z2, Z1), D1);
        G = fma2(bc2(-0.5f), sub(mA, carry), D1);
        carry = mA;
      } else if (SCHEME == LBM_SCHEME_UPWIND2) {
        G = mul(half, sub(fma2(bc2(4.f), Z1, mul(bc2(-3.f), B)), Z2));
      } else {
        G = D1;
      }
      acc(G, false);
    }
    if (i <= 6) nsum(add(H, Z1));
  }
  const float keep = i == 0 ? m.keep0 : (i <= 6 ? m.keep1 : m.keep2);
  const float kk = i == 0 ? 0.f : (i <= 6 ? m.k1 : m.k2);
  const float lam = i == 0 ? m.lam0 : (i <= 6 ? m.lam1 : 0.f);
  // keep_i f + (dt/tau) f^eq.  R1 (dt = tau): dt/tau = 1, so the product with
  // it is f^eq exactly, and keep_2 = 1 - dt/tau = 0 for the diagonal
  // velocities, whose sum is then f^eq exactly: bitwise the general form
  float2 o;
  if (R1) o = i >= 7 ? fe : fma2(bc2(keep), B, fe);
  else o = fma2(bc2(keep), B, mul(bc2(m.dt_tau), fe));
  if (i != 0) o = fma2(bc2(cneg ? kk : -kk), conv, o);
  if (i <= 6) o = fma2(bc2(lam), S, o);
  return o;
}

// Initial z-interface minmod of field i for a unit starting at plane k = 0
// (NND): the interface below plane 0 from planes -2, -1 (h2, h1), 0 (fc) and,
// for v_z < 0, plane 1 (fz1).
__device__ __forceinline__ float2 carry0(int i, float2 h2, float2 h1, float2 fc, float2 fz1) {
  const int sz = vsign(i, 2);
  if (sz > 0) return mmc2(sub(h1, h2), sub(fc, h1));
  if (sz < 0) return mmc2(sub(fz1, fc), sub(fc, h1));
  return make_float2(0.f, 0.f);
}

// The two layers outside an x face from the boundary cell c0 (next to the
// face) and its neighbour c1 (Sec. 4(2)): g1 next to the face, g2 outside it.
__device__ __forceinline__ void x_face_layers(const Model<float>& m, int kind, const float c0[NV], const float c1[NV],
                                              float g1[NV], float g2[NV]) {
  float M0[5], M1[5], G1[5], G2[5];
  lbm::moments(m, c0, M0[0], M0[1], M0[2], M0[3], M0[4]);
  if (kind == LBM_BC_EXTRAPOLATE) {
    lbm::moments(m, c1, M1[0], M1[1], M1[2], M1[3], M1[4]);
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
  lbm::equilibrium(m, G1[0], G1[1], G1[2], G1[3], G1[4], g1);
  lbm::equilibrium(m, G2[0], G2[1], G2[2], G2[3], G2[4], g2);
}

}  // namespace pm
}  // namespace lbm
