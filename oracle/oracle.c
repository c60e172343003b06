/*
 * FP64 CPU oracle of the D3V15 finite-difference lattice Boltzmann step of
 * Chen, Xu, Zhang & Li, "Three-Dimensional Lattice Boltzmann Model for
 * High-Speed Compressible Flows" (arXiv:1010.4135).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only tests/, the smoke()
 * entry of __graft_entry__ and the CPU-baseline leg of bench.py may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is double precision and evaluated in the order the paper writes
 * it.  The build uses -ffp-contract=off so no multiply-add is fused.
 *
 * Field layout of every f array passed in or out: f[i][z][y][x], i = 0..14
 * (the paper's i = 1..15), x fastest, interior cells only, nx*ny*nz per field.
 * Macroscopic fields rho, T are [z][y][x]; u is [3][z][y][x].
 *
 * Parity of each function with the paper:
 *   oracle_velocities  Sec. 2, discrete velocity set and eta_i (Eq. "vv")
 *   oracle_feq         Sec. 2, equilibrium (Eq. "eq") with A_i, B_i, D_i
 *   oracle_moments     Sec. 2, moment relations (e1)-(e3) read as definitions
 *   oracle_step        Sec. 3: NND flux (Eq. "nnd" and the flux definitions
 *                      under it), minmod, the extra dissipation term (Eq.
 *                      "lp"), BGK relaxation (Eq. 1) and a first-order
 *                      forward time step; boundary layers of Sec. 4(2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 15

/* Boundary kinds of the two layers outside each face. */
enum { OBC_PERIODIC = 0, OBC_FIXED = 1, OBC_EXTRAPOLATE = 2, OBC_REFLECT = 3 };
/* Convection schemes: the paper's NND, and the two upwind schemes the paper
 * compares it with (Sec. 3 first paragraph; Fig. 6) and linearises (G with
 * alpha~ = beta~ = 0 is first-order upwind). */
enum { OSCHEME_NND = 0, OSCHEME_UPWIND2 = 1, OSCHEME_UPWIND1 = 2 };

typedef struct {
  int32_t nx, ny, nz;
  int32_t bc_lo[3], bc_hi[3];
  double fixed_lo[3][5], fixed_hi[3][5]; /* (rho, u1, u2, u3, T) per face */
  double c1, c2, eta0, gamma;
  double tau, dt, dx;
  int32_t scheme;
  int32_t dissipation; /* 1: lambda_i of Eq. "lp"; 0: no extra term */
} oracle_cfg;

/* ---------------------------------------------------------------- model */

/* Discrete velocities and eta_i (Sec. 2): i=1 rest; i=2..7 c1 along +-x,
 * +-y, +-z; i=8..15 c2/sqrt(3) (+-1,+-1,+-1).  Order inside each group:
 * +x,-x,+y,-y,+z,-z, then the sign triples (+++,++-,+-+,+--,-++,-+-,--+,---). */
void oracle_velocities(const oracle_cfg* c, double v[NV][3], double eta[NV]) {
  for (int i = 0; i < NV; ++i) { v[i][0] = v[i][1] = v[i][2] = 0.0; eta[i] = 0.0; }
  eta[0] = c->eta0;
  for (int a = 0; a < 3; ++a) {
    v[1 + 2 * a][a] = c->c1;
    v[2 + 2 * a][a] = -c->c1;
  }
  double s = c->c2 / sqrt(3.0);
  for (int k = 0; k < 8; ++k) {
    v[7 + k][0] = (k & 4) ? -s : s;
    v[7 + k][1] = (k & 2) ? -s : s;
    v[7 + k][2] = (k & 1) ? -s : s;
  }
}

static double gas_b(const oracle_cfg* c) { return 2.0 / (c->gamma - 1.0); }

/* Equilibrium f_i^eq = rho (A_i + B_i v_ia u_a + D_i (u_a v_ia)^2), Eq. "eq"
 * with the three-case A_i, B_i, D_i printed beneath it (R = 1). */
void oracle_feq(const oracle_cfg* c, double rho, const double u[3], double T, double feq[NV]) {
  double v[NV][3], eta[NV];
  oracle_velocities(c, v, eta);
  const double b = gas_b(c);
  const double c1 = c->c1, c2 = c->c2, e0 = c->eta0;
  const double c12 = c1 * c1, c22 = c2 * c2;
  const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < NV; ++i) {
    double A, B, D;
    if (i == 0) {
      A = (b - 3.0) / (e0 * e0) * T;
      B = 0.0;
      D = 0.0;
    } else if (i <= 6) {
      A = 1.0 / (6.0 * (c12 - c22)) * (-c22 + ((b - 3.0) * c22 / (e0 * e0) + 3.0) * T + c22 / c12 * usq);
      B = (-c22 + (b + 2.0) * T + usq) / (2.0 * c12 * (c12 - c22));
      D = 1.0 / (2.0 * c12 * c12);
    } else {
      A = 1.0 / (8.0 * (c22 - c12)) *
          (-c12 + ((b - 3.0) * c12 / (e0 * e0) + 3.0) * T + (3.0 * c12 - c22) / (2.0 * c22) * usq);
      B = 3.0 * (-c12 + (b + 2.0) * T + usq) / (8.0 * c22 * (c22 - c12));
      D = 9.0 / (16.0 * c22 * c22);
    }
    double vu = v[i][0] * u[0] + v[i][1] * u[1] + v[i][2] * u[2];
    feq[i] = rho * (A + B * vu + D * vu * vu);
  }
}

/* Moments of one node's 15 values (Sec. 2, (e1)-(e3) taken as the
 * definitions of rho, rho u and the energy): out = (rho, u1, u2, u3, T, E)
 * with E = sum f_i (v_i^2 + eta_i^2) and T = (E/rho - u^2)/b. */
void oracle_moments(const oracle_cfg* c, const double f[NV], double out[6]) {
  double v[NV][3], eta[NV];
  oracle_velocities(c, v, eta);
  double rho = 0.0, m[3] = {0.0, 0.0, 0.0}, E = 0.0;
  for (int i = 0; i < NV; ++i) {
    rho += f[i];
    for (int a = 0; a < 3; ++a) m[a] += f[i] * v[i][a];
    double vsq = v[i][0] * v[i][0] + v[i][1] * v[i][1] + v[i][2] * v[i][2];
    E += f[i] * (vsq + eta[i] * eta[i]);
  }
  double u0 = m[0] / rho, u1 = m[1] / rho, u2 = m[2] / rho;
  double T = (E / rho - (u0 * u0 + u1 * u1 + u2 * u2)) / gas_b(c);
  out[0] = rho; out[1] = u0; out[2] = u1; out[3] = u2; out[4] = T; out[5] = E;
}

/* ------------------------------------------------------------- grid access */

/* Read-only view of a field array: element (i, x, y, z), with interior
 * coordinates x, y, z, sits at d[i*si + (z+off)*sz + (y+off)*sy + (x+off)].
 * off = 2 for the padded working copy, 0 for a caller's interior array. */
typedef struct {
  const double* d;
  size_t si, sz, sy;
  int off;
} view;

static double vget(const view* V, int i, int x, int y, int z) {
  return V->d[(size_t)i * V->si + (size_t)(z + V->off) * V->sz + (size_t)(y + V->off) * V->sy + (size_t)(x + V->off)];
}

static view interior_view(const oracle_cfg* c, const double* f) {
  view V;
  V.d = f;
  V.sy = (size_t)c->nx;
  V.sz = V.sy * c->ny;
  V.si = V.sz * c->nz;
  V.off = 0;
  return V;
}

static int wrap(int k, int n) {
  int r = k % n;
  return r < 0 ? r + n : r;
}

/* Macroscopic (rho, u1, u2, u3, T) of one interior node. */
static void node_macros(const oracle_cfg* c, const view* V, int x, int y, int z, double m[5]) {
  double f[NV], out[6];
  for (int i = 0; i < NV; ++i) f[i] = vget(V, i, x, y, z);
  oracle_moments(c, f, out);
  for (int k = 0; k < 5; ++k) m[k] = out[k];
}

/* Macros of the two layers outside one non-periodic face at the cross
 * position pos (pos[axis] is ignored).  Sec. 4(2): fixed values in both
 * layers; linear extrapolation g1 = 2 m0 - m1, g2 = 2 g1 - m0 on rho, T and
 * u; reflection with the wall layer taking (rho, T, u_t) of the last interior
 * node and u_n = 0, and the outer layer mirroring the last interior node with
 * u_n negated.  G1 is the layer next to the face, G2 the outer one. */
static void ghost_macros(const oracle_cfg* c, const view* V, int axis, int hi, const int pos[3],
                         double G1[5], double G2[5]) {
  const int n[3] = {c->nx, c->ny, c->nz};
  const int kind = hi ? c->bc_hi[axis] : c->bc_lo[axis];
  const int m0 = hi ? n[axis] - 1 : 0; /* last interior node */
  const int m1 = hi ? n[axis] - 2 : 1; /* the one before it  */
  if (kind == OBC_FIXED) {
    const double* fx = hi ? c->fixed_hi[axis] : c->fixed_lo[axis];
    for (int k = 0; k < 5; ++k) G1[k] = G2[k] = fx[k];
  } else if (kind == OBC_EXTRAPOLATE) {
    double M0[5], M1[5];
    int p0[3] = {pos[0], pos[1], pos[2]}, p1[3] = {pos[0], pos[1], pos[2]};
    p0[axis] = m0;
    p1[axis] = m1;
    node_macros(c, V, p0[0], p0[1], p0[2], M0);
    node_macros(c, V, p1[0], p1[1], p1[2], M1);
    for (int k = 0; k < 5; ++k) {
      G1[k] = 2.0 * M0[k] - M1[k];
      G2[k] = 2.0 * G1[k] - M0[k];
    }
  } else { /* OBC_REFLECT */
    double M0[5];
    int p0[3] = {pos[0], pos[1], pos[2]};
    p0[axis] = m0;
    node_macros(c, V, p0[0], p0[1], p0[2], M0);
    for (int k = 0; k < 5; ++k) G1[k] = G2[k] = M0[k];
    G1[1 + axis] = 0.0;
    G2[1 + axis] = -M0[1 + axis];
  }
}

/* f_i at any node within two layers of the interior, from interior data:
 * periodic faces wrap, the others give f^eq of the ghost macros.  Nodes
 * outside the interior along two or more axes (edges, corners) are never
 * read by the star stencil and are not defined. */
static double fetch(const oracle_cfg* c, const view* V, int i, int x, int y, int z) {
  const int n[3] = {c->nx, c->ny, c->nz};
  int q[3] = {x, y, z};
  for (int a = 0; a < 3; ++a) {
    if (q[a] >= 0 && q[a] < n[a]) continue;
    const int hi = q[a] >= n[a];
    const int kind = hi ? c->bc_hi[a] : c->bc_lo[a];
    if (kind == OBC_PERIODIC) {
      q[a] = wrap(q[a], n[a]);
      return vget(V, i, q[0], q[1], q[2]);
    }
    double G1[5], G2[5], feq[NV];
    ghost_macros(c, V, a, hi, q, G1, G2);
    const int outer = hi ? (q[a] == n[a] + 1) : (q[a] == -2);
    const double* G = outer ? G2 : G1;
    const double u[3] = {G[1], G[2], G[3]};
    oracle_feq(c, G[0], u, G[4], feq);
    return feq[i];
  }
  return vget(V, i, q[0], q[1], q[2]);
}

/* ------------------------------------------------------------ convection */

static double sign_of(double x) { return (x > 0.0) - (x < 0.0); }

/* minmod(X, Y) = 1/2 min(|X|, |Y|) [Sign(X) + Sign(Y)]  (Sec. 3) */
static double minmod(double X, double Y) {
  return 0.5 * fmin(fabs(X), fabs(Y)) * (sign_of(X) + sign_of(Y));
}

/* Numerical flux h_{I+1/2} from the four values f_{I-1}, f_I, f_{I+1},
 * f_{I+2} along one axis, with the split f^+- = (v +- |v|) f / 2 (Sec. 3).
 * NND: h = f^L + f^R, f^L = f^+_I + minmod(df^+_{I+1/2}, df^+_{I-1/2}) / 2,
 *      f^R = f^-_{I+1} - minmod(df^-_{I+1/2}, df^-_{I+3/2}) / 2.
 * UPWIND2 (second-order upwind): h = (3 f^+_I - f^+_{I-1})/2 + (3 f^-_{I+1} - f^-_{I+2})/2.
 * UPWIND1 (first-order upwind):  h = f^+_I + f^-_{I+1}. */
static double flux(int scheme, double v, double fm1, double f0, double f1, double f2) {
  const double wp = 0.5 * (v + fabs(v)), wm = 0.5 * (v - fabs(v));
  const double pm1 = wp * fm1, p0 = wp * f0, p1 = wp * f1;
  const double m0 = wm * f0, m1 = wm * f1, m2 = wm * f2;
  if (scheme == OSCHEME_UPWIND1) return p0 + m1;
  if (scheme == OSCHEME_UPWIND2) return 0.5 * (3.0 * p0 - pm1) + 0.5 * (3.0 * m1 - m2);
  const double fL = p0 + 0.5 * minmod(p1 - p0, p0 - pm1);
  const double fR = m1 - 0.5 * minmod(m1 - m0, m2 - m1);
  return fL + fR;
}

/* -------------------------------------------------------------------- step */

static int cfg_valid(const oracle_cfg* c) {
  if (c->nx < 1 || c->ny < 1 || c->nz < 1) return 0;
  const int n[3] = {c->nx, c->ny, c->nz};
  for (int a = 0; a < 3; ++a) {
    if ((c->bc_lo[a] == OBC_PERIODIC) != (c->bc_hi[a] == OBC_PERIODIC)) return 0;
    if ((c->bc_lo[a] == OBC_EXTRAPOLATE || c->bc_hi[a] == OBC_EXTRAPOLATE) && n[a] < 2) return 0;
  }
  return 1;
}

/* The new values of one node from its stencil S[i][a][k] = f_i at offset
 * k-2 along axis a (S[i][a][2] is the node itself):
 *   f_i^{n+1} = f_i^n + dt [ -(f_i - f_i^eq)/tau
 *                            - sum_a (h_{i,I+1/2} - h_{i,I-1/2}) / dx
 *                            + lambda_i sum_a (f_{I+1} - 2 f_I + f_{I-1}) / dx^2 ]
 * (Eq. 1 with Eq. "lp", the NND flux of Eq. "nnd", forward Euler in time). */
static void update_node(const oracle_cfg* c, const double S[NV][3][5], double out[NV]) {
  double v[NV][3], eta[NV], lambda[NV];
  oracle_velocities(c, v, eta);
  for (int i = 0; i < NV; ++i) {
    if (!c->dissipation) lambda[i] = 0.0;
    else if (i == 0) lambda[i] = c->c1 * c->dx;
    else if (i <= 6) lambda[i] = c->c1 * c->dx / 10.0;
    else lambda[i] = 0.0;
  }
  double fc[NV], mac[6], feq[NV];
  for (int i = 0; i < NV; ++i) fc[i] = S[i][0][2];
  oracle_moments(c, fc, mac);
  const double u[3] = {mac[1], mac[2], mac[3]};
  oracle_feq(c, mac[0], u, mac[4], feq);
  for (int i = 0; i < NV; ++i) {
    double conv = 0.0, lap = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double* s = S[i][a];
      double hp = flux(c->scheme, v[i][a], s[1], s[2], s[3], s[4]); /* h_{I+1/2} */
      double hm = flux(c->scheme, v[i][a], s[0], s[1], s[2], s[3]); /* h_{I-1/2} */
      conv += (hp - hm) / c->dx;
      lap += (s[3] - 2.0 * s[2] + s[1]) / (c->dx * c->dx);
    }
    double rhs = -(fc[i] - feq[i]) / c->tau - conv + lambda[i] * lap;
    out[i] = fc[i] + c->dt * rhs;
  }
}

/* Working copy with two boundary layers on every side: the paper's node
 * numbering 0, 1, ..., NX, NX+1 (Sec. 4(2)); edges and corners stay NaN. */
typedef struct {
  double* d;
  view V;
} padded;

static int padded_alloc(const oracle_cfg* c, padded* P) {
  const size_t px = (size_t)c->nx + 4, py = (size_t)c->ny + 4, pz = (size_t)c->nz + 4;
  const size_t cnt = (size_t)NV * px * py * pz;
  P->d = (double*)malloc(cnt * sizeof(double));
  if (!P->d) return 0;
  for (size_t k = 0; k < cnt; ++k) P->d[k] = NAN;
  P->V.d = P->d;
  P->V.sy = px;
  P->V.sz = px * py;
  P->V.si = px * py * pz;
  P->V.off = 2;
  return 1;
}

static double* pref(padded* P, int i, int x, int y, int z) {
  return P->d + ((size_t)i * P->V.si + (size_t)(z + 2) * P->V.sz + (size_t)(y + 2) * P->V.sy + (size_t)(x + 2));
}

/* Copy the interior in, then fill the two layers outside every face. */
static void build_padded(const oracle_cfg* c, padded* P, const double* f) {
  const int n[3] = {c->nx, c->ny, c->nz};
  const view I = interior_view(c, f);
#pragma omp parallel for collapse(2) schedule(static)
  for (int i = 0; i < NV; ++i)
    for (int z = 0; z < n[2]; ++z)
      for (int y = 0; y < n[1]; ++y)
        for (int x = 0; x < n[0]; ++x) *pref(P, i, x, y, z) = vget(&I, i, x, y, z);
  for (int a = 0; a < 3; ++a) {
    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    for (int hi = 0; hi < 2; ++hi)
      for (int s2 = 0; s2 < n[a2]; ++s2)
        for (int s1 = 0; s1 < n[a1]; ++s1)
          for (int layer = 0; layer < 2; ++layer) {
            int q[3];
            q[a1] = s1;
            q[a2] = s2;
            q[a] = hi ? n[a] + layer : -1 - layer;
            for (int i = 0; i < NV; ++i) *pref(P, i, q[0], q[1], q[2]) = fetch(c, &I, i, q[0], q[1], q[2]);
          }
  }
}

static void gather_stencil(const view* V, int x, int y, int z, double S[NV][3][5]) {
  for (int i = 0; i < NV; ++i)
    for (int a = 0; a < 3; ++a)
      for (int k = -2; k <= 2; ++k) {
        int q[3] = {x, y, z};
        q[a] += k;
        S[i][a][k + 2] = vget(V, i, q[0], q[1], q[2]);
      }
}

static void step_padded(const oracle_cfg* c, const padded* P, double* fout, int nthreads) {
  const int n[3] = {c->nx, c->ny, c->nz};
  const size_t nxy = (size_t)n[0] * n[1], ncell = nxy * n[2];
  (void)nthreads;
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
  for (int z = 0; z < n[2]; ++z) {
    for (int y = 0; y < n[1]; ++y) {
      for (int x = 0; x < n[0]; ++x) {
        double S[NV][3][5], out[NV];
        gather_stencil(&P->V, x, y, z, S);
        update_node(c, S, out);
        for (int i = 0; i < NV; ++i) fout[i * ncell + (size_t)z * nxy + (size_t)y * n[0] + x] = out[i];
      }
    }
  }
}

/* Advance f (interior, [15][nz][ny][nx]) by nsteps steps in place.
 * Returns 0 on success, -1 on an invalid configuration, -2 on no memory. */
int oracle_run(const oracle_cfg* c, double* f, int64_t nsteps, int nthreads) {
  if (!cfg_valid(c)) return -1;
  padded P;
  if (!padded_alloc(c, &P)) return -2;
  for (int64_t s = 0; s < nsteps; ++s) {
    build_padded(c, &P, f);
    step_padded(c, &P, f, nthreads);
  }
  free(P.d);
  return 0;
}

/* One step from fin into fout (distinct arrays). */
int oracle_step(const oracle_cfg* c, const double* fin, double* fout, int nthreads) {
  if (!cfg_valid(c)) return -1;
  padded P;
  if (!padded_alloc(c, &P)) return -2;
  build_padded(c, &P, fin);
  step_padded(c, &P, fout, nthreads);
  free(P.d);
  return 0;
}

/* One step evaluated only at ncells nodes (x, y, z triples in xyz), reading
 * the boundary layers on the fly: out[k][15] is the new state of node k. */
int oracle_step_nodes(const oracle_cfg* c, const double* f, int64_t ncells, const int32_t* xyz, double* out) {
  if (!cfg_valid(c)) return -1;
  for (int64_t k = 0; k < ncells; ++k) {
    const int x = xyz[3 * k], y = xyz[3 * k + 1], z = xyz[3 * k + 2];
    if (x < 0 || y < 0 || z < 0 || x >= c->nx || y >= c->ny || z >= c->nz) return -1;
  }
  const view I = interior_view(c, f);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < ncells; ++k) {
    const int x = xyz[3 * k], y = xyz[3 * k + 1], z = xyz[3 * k + 2];
    double S[NV][3][5];
    for (int i = 0; i < NV; ++i)
      for (int a = 0; a < 3; ++a)
        for (int d = -2; d <= 2; ++d) {
          int q[3] = {x, y, z};
          q[a] += d;
          S[i][a][d + 2] = fetch(c, &I, i, q[0], q[1], q[2]);
        }
    update_node(c, S, out + 15 * k);
  }
  return 0;
}

/* The padded working copy (two layers per face) as the step sees it:
 * out is [15][nz+4][ny+4][nx+4]; edges and corners are NaN. */
int oracle_padded(const oracle_cfg* c, const double* f, double* out) {
  if (!cfg_valid(c)) return -1;
  padded P;
  if (!padded_alloc(c, &P)) return -2;
  build_padded(c, &P, f);
  memcpy(out, P.d, sizeof(double) * (size_t)NV * (c->nx + 4) * (c->ny + 4) * (c->nz + 4));
  free(P.d);
  return 0;
}

/* f = f^eq(rho, u, T) at every interior node. */
void oracle_init(const oracle_cfg* c, const double* rho, const double* u, const double* T, double* f) {
  const int64_t ncell = (int64_t)c->nx * c->ny * c->nz;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < ncell; ++k) {
    double uu[3] = {u[k], u[ncell + k], u[2 * ncell + k]}, feq[NV];
    oracle_feq(c, rho[k], uu, T[k], feq);
    for (int i = 0; i < NV; ++i) f[i * ncell + k] = feq[i];
  }
}

/* Macroscopic fields of every interior node. */
void oracle_macros(const oracle_cfg* c, const double* f, double* rho, double* u, double* T) {
  const int64_t ncell = (int64_t)c->nx * c->ny * c->nz;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < ncell; ++k) {
    double fc[NV], out[6];
    for (int i = 0; i < NV; ++i) fc[i] = f[i * ncell + k];
    oracle_moments(c, fc, out);
    rho[k] = out[0];
    u[k] = out[1];
    u[ncell + k] = out[2];
    u[2 * ncell + k] = out[3];
    T[k] = out[4];
  }
}

/* Global mass, momentum and energy: out = (sum rho, sum rho u1, sum rho u2,
 * sum rho u3, sum E), summed node by node in storage order. */
void oracle_conserved(const oracle_cfg* c, const double* f, double out[5]) {
  const size_t ncell = (size_t)c->nx * c->ny * c->nz;
  double v[NV][3], eta[NV];
  oracle_velocities(c, v, eta);
  for (int k = 0; k < 5; ++k) out[k] = 0.0;
  for (size_t k = 0; k < ncell; ++k) {
    for (int i = 0; i < NV; ++i) {
      double fi = f[i * ncell + k];
      double vsq = v[i][0] * v[i][0] + v[i][1] * v[i][1] + v[i][2] * v[i][2];
      out[0] += fi;
      out[1] += fi * v[i][0];
      out[2] += fi * v[i][1];
      out[3] += fi * v[i][2];
      out[4] += fi * (vsq + eta[i] * eta[i]);
    }
  }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
