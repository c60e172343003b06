// Von Neumann amplification service (Sec. 3) for choosing run parameters.
//
// For a perturbation F exp(i k.x) of a uniform state (rho, u, T), one step
// multiplies F by the 15 x 15 complex matrix
//   G_ij = (1 - dt/tau - sum_a v_ia dt/dx phi_ia
//           + lambda_i dt sum_a (2 cos(k_a dx) - 2)/dx^2) delta_ij + dt/tau dfeq_i/df_j,
//   phi_ia = 1 - exp(-i k_a dx) for v_ia >= 0, exp(i k_a dx) - 1 otherwise
// (the paper's G with alpha~ = beta~ = 0), with the equilibrium Jacobian by
// the chain rule through (rho, u, T):
//   d rho/df_j = 1,  d u_a/df_j = (v_ja - u_a)/rho,
//   d T/df_j = (|v_j - u|^2 + eta_j^2 - b T)/(b rho),
// and the partial derivatives of f^eq_i = rho (A_i + B_i w_i + D_i w_i^2),
// w_i = v_i . u, with A_i, B_i affine in T and |u|^2 per velocity shell
// (Eq. "eq").  The service returns, per parameter set, the largest spectral
// radius max |omega| over a batch of states, wave-vector directions and
// wave numbers k dx = pi q / nk (q = 1 .. nk): the paper's stability measure.
//
// One thread per matrix.  The eigenvalues come from a Householder reduction
// to upper Hessenberg form followed by the single-shift complex QR
// iteration with Wilkinson shifts, deflation at negligible subdiagonal
// entries and an exceptional shift after 10 and 20 iterations without one
// (the practical QR algorithm of Golub and Van Loan, Sec. 7.5, here without
// accumulating the transformations: only eigenvalues are needed, so each QR
// step acts on the unreduced diagonal block alone).  A matrix that has not
// converged after 30 n iterations reports +inf, which the caller reads as
// unstable.  The matrices live in shared memory, interleaved by thread.
#include <cmath>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int VN = NV;              // matrix order
constexpr int VN_THREADS = 32;      // matrices per block
constexpr int VN_PARAMS = 7;        // c1, c2, eta0, gamma, dt, tau, dx
constexpr int VN_MAX_ITER = 30 * VN;

struct cd {
  double re, im;
};
__device__ __forceinline__ cd mk(double r, double i) { return {r, i}; }
__device__ __forceinline__ cd operator+(cd a, cd b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cd operator-(cd a, cd b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cd operator*(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cd operator*(double s, cd a) { return {s * a.re, s * a.im}; }
__device__ __forceinline__ cd cconj(cd a) { return {a.re, -a.im}; }
__device__ __forceinline__ double cabs(cd a) { return hypot(a.re, a.im); }
__device__ __forceinline__ double cabs1(cd a) { return fabs(a.re) + fabs(a.im); }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__device__ __forceinline__ cd csqrt_(cd a) {
  const double r = cabs(a);
  if (r == 0.0) return {0.0, 0.0};
  const double t = sqrt(0.5 * (r + fabs(a.re)));
  return a.re >= 0.0 ? cd{t, a.im / (2.0 * t)} : cd{fabs(a.im) / (2.0 * t), copysign(t, a.im)};
}

// Matrix of this thread: element (r, c) at m[(r * VN + c) * VN_THREADS].
struct Mat {
  cd* m;
  __device__ cd& at(int r, int c) const { return m[(r * VN + c) * VN_THREADS]; }
};

// The discrete velocities (Sec. 2) in the library's order: 0 rest; 1..6 +-c1
// along x, y, z; 7..14 (c2/sqrt 3)(sx, sy, sz), signs +++, ++-, ..., ---.
__device__ void velocity(int i, double c1, double s, double v[3]) {
  v[0] = v[1] = v[2] = 0.0;
  if (i == 0) return;
  if (i <= 6) {
    v[(i - 1) / 2] = ((i - 1) % 2 == 0) ? c1 : -c1;
    return;
  }
  const int k = i - 7;
  v[0] = (k & 4) ? -s : s;
  v[1] = (k & 2) ? -s : s;
  v[2] = (k & 1) ? -s : s;
}

// Per-velocity coefficients of Eq. "eq": A = A0 + AT T + AU u^2, B = B0 + BT T
// + BU u^2, D.
__device__ void shell(int i, double c1, double c2, double eta0, double b, double co[7]) {
  const double c12 = c1 * c1, c22 = c2 * c2, e2 = eta0 * eta0;
  if (i == 0) {
    co[0] = 0.0; co[1] = (b - 3.0) / e2; co[2] = 0.0; co[3] = co[4] = co[5] = co[6] = 0.0;
  } else if (i <= 6) {
    const double ka = 1.0 / (6.0 * (c12 - c22)), kb = 1.0 / (2.0 * c12 * (c12 - c22));
    co[0] = -c22 * ka; co[1] = ((b - 3.0) * c22 / e2 + 3.0) * ka; co[2] = c22 / c12 * ka;
    co[3] = -c22 * kb; co[4] = (b + 2.0) * kb; co[5] = kb; co[6] = 1.0 / (2.0 * c12 * c12);
  } else {
    const double kd = 1.0 / (8.0 * (c22 - c12)), ke = 3.0 / (8.0 * c22 * (c22 - c12));
    co[0] = -c12 * kd; co[1] = ((b - 3.0) * c12 / e2 + 3.0) * kd; co[2] = (3.0 * c12 - c22) / (2.0 * c22) * kd;
    co[3] = -c12 * ke; co[4] = (b + 2.0) * ke; co[5] = ke; co[6] = 9.0 / (16.0 * c22 * c22);
  }
}

// G(k) of the state st = (rho, u1, u2, u3, T) and parameters p into M.
__device__ void build_g(const Mat& M, const double* st, const double* p, const double kv[3], int dissipation) {
  const double c1 = p[0], c2 = p[1], eta0 = p[2], gamma = p[3], dt = p[4], tau = p[5], dx = p[6];
  const double b = 2.0 / (gamma - 1.0), s = c2 / sqrt(3.0);
  const double rho = st[0], u[3] = {st[1], st[2], st[3]}, T = st[4];
  const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double r = dt / tau;
  // column factors of the chain rule: d u_a/df_j and d T/df_j
  double du[VN][3], dT[VN];
  for (int j = 0; j < VN; ++j) {
    double vj[3];
    velocity(j, c1, s, vj);
    double rel2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      du[j][a] = (vj[a] - u[a]) / rho;
      rel2 += (vj[a] - u[a]) * (vj[a] - u[a]);
    }
    const double eta = j == 0 ? eta0 : 0.0;
    dT[j] = (rel2 + eta * eta - b * T) / (b * rho);
  }
  for (int i = 0; i < VN; ++i) {
    double vi[3], co[7];
    velocity(i, c1, s, vi);
    shell(i, c1, c2, eta0, b, co);
    const double w = vi[0] * u[0] + vi[1] * u[1] + vi[2] * u[2];
    const double A = co[0] + co[1] * T + co[2] * usq, B = co[3] + co[4] * T + co[5] * usq, D = co[6];
    const double f_rho = A + B * w + D * w * w;
    const double f_T = rho * (co[1] + co[4] * w);
    double f_u[3];
    for (int a = 0; a < 3; ++a) f_u[a] = rho * ((2.0 * co[2] + 2.0 * co[5] * w) * u[a] + (B + 2.0 * D * w) * vi[a]);
    for (int j = 0; j < VN; ++j) {
      const double J = f_rho + f_T * dT[j] + f_u[0] * du[j][0] + f_u[1] * du[j][1] + f_u[2] * du[j][2];
      M.at(i, j) = mk(r * J, 0.0);
    }
    // diagonal: relaxation, convection (first-order upwind phase), dissipation
    const double lam = !dissipation ? 0.0 : (i == 0 ? c1 * dx : (i <= 6 ? c1 * dx / 10.0 : 0.0));
    cd d = mk(1.0 - r, 0.0);
    for (int a = 0; a < 3; ++a) {
      const double th = kv[a] * dx, cs = cos(th), sn = sin(th);
      // phi = 1 - e^{-i th} = (1 - cos th) + i sin th ; e^{i th} - 1 = (cos th - 1) + i sin th
      const cd phi = vi[a] >= 0.0 ? mk(1.0 - cs, sn) : mk(cs - 1.0, sn);
      d = d - (vi[a] * dt / dx) * phi;
      d = d + mk(lam * dt * (2.0 * cs - 2.0) / (dx * dx), 0.0);
    }
    M.at(i, i) = M.at(i, i) + d;
  }
}

// Spectral radius of M (destroyed), or +inf if the QR iteration does not converge.
__device__ double spectral_radius(const Mat& M) {
  const int n = VN;
  // Householder reduction to upper Hessenberg form (similarity, eigenvalues kept)
  for (int k = 0; k + 2 < n; ++k) {
    double tail = 0.0;  // squared norm below the subdiagonal
    for (int i = k + 2; i < n; ++i) tail += M.at(i, k).re * M.at(i, k).re + M.at(i, k).im * M.at(i, k).im;
    if (tail == 0.0) continue;  // the column is already in Hessenberg form
    const double alpha2 = tail + M.at(k + 1, k).re * M.at(k + 1, k).re + M.at(k + 1, k).im * M.at(k + 1, k).im;
    const double alpha = sqrt(alpha2);
    const cd x0 = M.at(k + 1, k);
    const double ax0 = cabs(x0);
    const cd phase = ax0 > 0.0 ? mk(x0.re / ax0, x0.im / ax0) : mk(1.0, 0.0);
    // v = x + phase alpha e1 (stored in column k below the diagonal), beta = 2 / |v|^2
    const cd v0 = x0 + alpha * phase;
    M.at(k + 1, k) = v0;
    const double vn2 = tail + v0.re * v0.re + v0.im * v0.im;
    const double beta = 2.0 / vn2;
    for (int j = k + 1; j < n; ++j) {  // left: rows k+1..n-1 of columns k+1..n-1
      cd sum = mk(0.0, 0.0);
      for (int i = k + 1; i < n; ++i) sum = sum + cconj(M.at(i, k)) * M.at(i, j);
      sum = beta * sum;
      for (int i = k + 1; i < n; ++i) M.at(i, j) = M.at(i, j) - M.at(i, k) * sum;
    }
    for (int r = 0; r < n; ++r) {  // right: columns k+1..n-1 of every row
      cd sum = mk(0.0, 0.0);
      for (int i = k + 1; i < n; ++i) sum = sum + M.at(r, i) * M.at(i, k);
      sum = beta * sum;
      for (int i = k + 1; i < n; ++i) M.at(r, i) = M.at(r, i) - sum * cconj(M.at(i, k));
    }
    // the reflected column: -phase alpha e1
    M.at(k + 1, k) = (-alpha) * phase;
    for (int i = k + 2; i < n; ++i) M.at(i, k) = mk(0.0, 0.0);
  }
  // shifted QR on the unreduced diagonal blocks, eigenvalues only.  A
  // subdiagonal entry is negligible below ulp times its diagonal neighbours
  // or ulp times the matrix norm: the iteration's backward error is of that
  // size anyway, and without the norm floor a cluster of tiny eigenvalues
  // (those of G for dt = tau are O(Courant number)) is never split off
  const double ulp = 2.220446049250313e-16;
  double nrm = 0.0;
  for (int r = 0; r < n; ++r)
    for (int c = r > 0 ? r - 1 : 0; c < n; ++c) nrm = fmax(nrm, cabs1(M.at(r, c)));
  const double floor_small = ulp * nrm;
  double radius = 0.0;
  int hi = n - 1, its = 0, total = 0;
  double gc[VN];
  cd gs[VN];
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      const double tst = cabs1(M.at(l - 1, l - 1)) + cabs1(M.at(l, l));
      if (cabs1(M.at(l, l - 1)) <= fmax(ulp * tst, floor_small)) {
        M.at(l, l - 1) = mk(0.0, 0.0);
        break;
      }
      --l;
    }
    if (l == hi) {  // a 1 x 1 block: an eigenvalue
      const double e = cabs(M.at(hi, hi));
      if (!(e <= 1e300)) return INFINITY;  // non-finite: reported as unstable
      radius = fmax(radius, e);
      --hi;
      its = 0;
      continue;
    }
    if (++total > VN_MAX_ITER) return INFINITY;
    ++its;
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer its last entry
    const cd a = M.at(hi - 1, hi - 1), bq = M.at(hi - 1, hi), c = M.at(hi, hi - 1), d = M.at(hi, hi);
    cd mu;
    if (its == 10 || its == 20) {  // exceptional shift
      mu = d + mk(0.75 * cabs1(c), 0.0);
    } else {
      const cd half = 0.5 * (a - d);
      const cd disc = csqrt_(half * half + bq * c);
      const cd m1 = d + half + disc, m2 = d + half - disc;
      mu = cabs1(m1 - d) <= cabs1(m2 - d) ? m1 : m2;
    }
    for (int j = l; j <= hi; ++j) M.at(j, j) = M.at(j, j) - mu;
    for (int j = l; j < hi; ++j) {
      const cd x = M.at(j, j), y = M.at(j + 1, j);
      const double ax = cabs(x), rr = hypot(ax, cabs(y));
      double cg;
      cd sg;
      if (rr == 0.0) {
        cg = 1.0;
        sg = mk(0.0, 0.0);
      } else if (ax == 0.0) {
        cg = 0.0;
        sg = mk(1.0, 0.0);
      } else {
        cg = ax / rr;
        sg = (1.0 / rr) * (mk(x.re / ax, x.im / ax) * cconj(y));
      }
      gc[j] = cg;
      gs[j] = sg;
      for (int col = j; col <= hi; ++col) {
        const cd t1 = M.at(j, col), t2 = M.at(j + 1, col);
        M.at(j, col) = cg * t1 + sg * t2;
        M.at(j + 1, col) = cg * t2 - cconj(sg) * t1;
      }
    }
    for (int j = l; j < hi; ++j) {
      const int rmax = j + 2 < hi ? j + 2 : hi;
      for (int r = l; r <= rmax; ++r) {
        const cd t1 = M.at(r, j), t2 = M.at(r, j + 1);
        M.at(r, j) = gc[j] * t1 + cconj(gs[j]) * t2;
        M.at(r, j + 1) = gc[j] * t2 - gs[j] * t1;
      }
    }
    for (int j = l; j <= hi; ++j) M.at(j, j) = M.at(j, j) + mu;
  }
  return radius;
}

// Item t of the batch: parameter set t / per_param, then state, direction and
// wave number; out[p] is the max over its items (atomic max of the bit
// patterns, which order like the values for non-negative doubles).
__global__ void __launch_bounds__(VN_THREADS)
    vn_kernel(const double* __restrict__ states, int nstates, const double* __restrict__ params, int nparams,
              const double* __restrict__ dirs, int ndirs, int nk, int dissipation,
              unsigned long long* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long per_param = (long long)nstates * ndirs * nk;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per_param * nparams) return;
  const int p = (int)(t / per_param);
  long long rem = t % per_param;
  const int s = (int)(rem / ((long long)ndirs * nk));
  rem %= (long long)ndirs * nk;
  const int d = (int)(rem / nk), q = (int)(rem % nk);
  const double* dv = dirs + 3 * d;
  const double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  const double dx = params[VN_PARAMS * p + 6];
  const double kdx = 3.141592653589793 * (q + 1) / nk;
  const double kv[3] = {dv[0] / dn * kdx / dx, dv[1] / dn * kdx / dx, dv[2] / dn * kdx / dx};
  Mat M{reinterpret_cast<cd*>(smem_raw) + threadIdx.x};
  build_g(M, states + 5 * s, params + VN_PARAMS * p, kv, dissipation);
  const double rad = spectral_radius(M);
  atomicMax(out + p, (unsigned long long)__double_as_longlong(rad));
}

constexpr size_t kVnSmem = (size_t)VN * VN * VN_THREADS * sizeof(cd);  // 115,200 bytes

}  // namespace

cudaError_t launch_vn_max_growth(const double* states, int nstates, const double* params, int nparams,
                                 const double* dirs, int ndirs, int nk, int dissipation, double* out,
                                 cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(vn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVnSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * nparams, st);
  if (e != cudaSuccess) return e;
  const long long items = (long long)nstates * ndirs * nk * nparams;
  const long long blocks = (items + VN_THREADS - 1) / VN_THREADS;
  vn_kernel<<<(unsigned)blocks, VN_THREADS, kVnSmem, st>>>(states, nstates, params, nparams, dirs, ndirs, nk,
                                                           dissipation, reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError();
}

}  // namespace lbm
