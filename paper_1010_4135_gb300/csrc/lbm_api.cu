// C ABI of the D3V15 FD-LB solver: argument checks, workspace carving,
// constant tables and kernel sequencing.  Declarations and the contract of
// every entry point are in include/lbm.h.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "lbm_internal.cuh"

using lbm::Layout;
using lbm::Model;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxRedBlocks = 1024;
constexpr size_t kRedBytes = (size_t)kMaxRedBlocks * 8 * sizeof(double);
constexpr size_t kStatusBytes = 256;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool grid_ok(const lbm_grid* g) {
  if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1) return false;
  if (g->nz > 65535 || g->ny > 65535 * 8) return false;
  const int n[3] = {g->nx, g->ny, g->nz};
  for (int a = 0; a < 3; ++a) {
    for (int h = 0; h < 2; ++h) {
      const int k = h ? g->bc_hi[a] : g->bc_lo[a];
      if (k < LBM_BC_PERIODIC || k > LBM_BC_REFLECT) return false;
      if (k == LBM_BC_EXTRAPOLATE && n[a] < 2) return false;
    }
    if ((g->bc_lo[a] == LBM_BC_PERIODIC) != (g->bc_hi[a] == LBM_BC_PERIODIC)) return false;
  }
  return true;
}

Layout make_layout(const lbm_grid* g) {
  Layout L;
  L.nx = g->nx;
  L.ny = g->ny;
  L.nz = g->nz;
  L.sx = (int)align_up((size_t)lbm::OX + (size_t)g->nx + 2, 32);
  L.plane = (long long)L.sx * (g->ny + 4);
  L.fs = (long long)align_up((size_t)L.plane * (size_t)(g->nz + 4), 64);
  return L;
}

size_t field_bytes(const Layout& L, int esz) { return align_up((size_t)lbm::NV * (size_t)L.fs * esz, kAlign); }

// Coefficients of Eq. "eq" regrouped per shell as affine functions of T and u^2.
Model<double> make_model(const lbm_vset* v, double tau, double dt, double dx, int dissipation) {
  Model<double> m;
  const double c1 = v->c1, c2 = v->c2, e0 = v->eta0;
  const double c12 = c1 * c1, c22 = c2 * c2, e02 = e0 * e0;
  const double b = 2.0 / (v->gamma - 1.0);
  m.c1 = c1;
  m.s = c2 / std::sqrt(3.0);
  m.eta0sq = e02;
  m.c1sq = c12;
  m.c2sq = c22;
  m.inv_b = 1.0 / b;
  m.AR = (b - 3.0) / e02;
  const double ka = 1.0 / (6.0 * (c12 - c22));
  m.Aa0 = -c22 * ka;
  m.AaT = ((b - 3.0) * c22 / e02 + 3.0) * ka;
  m.AaU = c22 / c12 * ka;
  const double kb = 1.0 / (2.0 * c12 * (c12 - c22));
  m.Ba0 = -c22 * kb;
  m.BaT = (b + 2.0) * kb;
  m.BaU = kb;
  m.Da = 1.0 / (2.0 * c12 * c12);
  const double kd = 1.0 / (8.0 * (c22 - c12));
  m.Ad0 = -c12 * kd;
  m.AdT = ((b - 3.0) * c12 / e02 + 3.0) * kd;
  m.AdU = (3.0 * c12 - c22) / (2.0 * c22) * kd;
  const double ke = 3.0 / (8.0 * c22 * (c22 - c12));
  m.Bd0 = -c12 * ke;
  m.BdT = (b + 2.0) * ke;
  m.BdU = ke;
  m.Dd = 9.0 / (16.0 * c22 * c22);
  m.dt_tau = dt / tau;
  m.k1 = c1 * dt / dx;
  m.k2 = m.s * dt / dx;
  // lambda_i (Eq. "lp"): c1 dx for the rest particle, c1 dx / 10 for the axis ones
  m.lam0 = dissipation ? c1 * dx * dt / (dx * dx) : 0.0;
  m.lam1 = dissipation ? c1 * dx / 10.0 * dt / (dx * dx) : 0.0;
  return m;
}

Model<float> to_float(const Model<double>& d) {
  Model<float> f;
  f.c1 = (float)d.c1; f.s = (float)d.s; f.eta0sq = (float)d.eta0sq; f.c1sq = (float)d.c1sq; f.c2sq = (float)d.c2sq;
  f.inv_b = (float)d.inv_b; f.AR = (float)d.AR;
  f.Aa0 = (float)d.Aa0; f.AaT = (float)d.AaT; f.AaU = (float)d.AaU;
  f.Ba0 = (float)d.Ba0; f.BaT = (float)d.BaT; f.BaU = (float)d.BaU; f.Da = (float)d.Da;
  f.Ad0 = (float)d.Ad0; f.AdT = (float)d.AdT; f.AdU = (float)d.AdU;
  f.Bd0 = (float)d.Bd0; f.BdT = (float)d.BdT; f.BdU = (float)d.BdU; f.Dd = (float)d.Dd;
  f.dt_tau = (float)d.dt_tau; f.k1 = (float)d.k1; f.k2 = (float)d.k2; f.lam0 = (float)d.lam0; f.lam1 = (float)d.lam1;
  return f;
}

}  // namespace

struct lbm_sim {
  int device;
  int prec, esz;
  Layout L;
  lbm_vset vset;
  double tau, dt, dx;
  int scheme, dissipation;
  Model<double> md;
  Model<float> mf;
  lbm::BcDesc bc;
  char* ws;
  size_t ws_bytes;
  void* fbuf[2];
  int cur;
  double* partials;
  unsigned* flags;
  unsigned* counter;
  double* result;
  cudaStream_t st;
  int64_t steps;
  int failed;
  int variant;          // LBM_VARIANT_* of the FP32 step
  int zchunk;           // 0 = automatic
  int num_sms;
  CUtensorMap tmap[2];  // FP32: TMA descriptors of the two f buffers
  // launch counting and event-pair timing
  int64_t launches[LBM_NKERNEL];
  double ms[LBM_NKERNEL];
  int timing;
  cudaEvent_t* ev;      // 2 * kRing events, or NULL
  int* ev_kind;         // kernel class of each ring slot
  int64_t ev_head, ev_tail;  // recorded / drained pair counters
};

namespace {

int fail(lbm_sim* s, cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  s->failed = 1;
  return LBM_ECUDA;
}

#define LBM_CK(sim, expr)                            \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return fail((sim), e_);   \
  } while (0)

int enter(lbm_sim* s) {
  if (!s) return LBM_EINVAL;
  if (s->failed) return LBM_ESTATE;
  if (cudaSetDevice(s->device) != cudaSuccess) return fail(s, cudaErrorInvalidDevice);
  return LBM_OK;
}

void* spare(lbm_sim* s) { return s->fbuf[s->cur ^ 1]; }

constexpr int kRing = 1024;

// Drain the oldest recorded pair (waits for its end event).
cudaError_t drain_one(lbm_sim* s) {
  const int slot = (int)(s->ev_tail % kRing);
  cudaError_t e = cudaEventSynchronize(s->ev[2 * slot + 1]);
  if (e != cudaSuccess) return e;
  float t = 0.f;
  e = cudaEventElapsedTime(&t, s->ev[2 * slot], s->ev[2 * slot + 1]);
  if (e != cudaSuccess) return e;
  s->ms[s->ev_kind[slot]] += t;
  s->ev_tail += 1;
  return cudaSuccess;
}

// Start of a launch of class `kind`: count it and, if timing, record the start event.
cudaError_t begin_launch(lbm_sim* s, int kind) {
  s->launches[kind] += 1;
  if (!s->timing) return cudaSuccess;
  if (s->ev_head - s->ev_tail >= kRing) {
    cudaError_t e = drain_one(s);
    if (e != cudaSuccess) return e;
  }
  const int slot = (int)(s->ev_head % kRing);
  s->ev_kind[slot] = kind;
  return cudaEventRecord(s->ev[2 * slot], s->st);
}

cudaError_t end_launch(lbm_sim* s, cudaError_t launch_status) {
  if (launch_status != cudaSuccess || !s->timing) return launch_status;
  const int slot = (int)(s->ev_head % kRing);
  s->ev_head += 1;
  return cudaEventRecord(s->ev[2 * slot + 1], s->st);
}

void free_events(lbm_sim* s) {
  if (s->ev) {
    for (int k = 0; k < 2 * kRing; ++k)
      if (s->ev[k]) cudaEventDestroy(s->ev[k]);
    free(s->ev);
    s->ev = nullptr;
  }
  free(s->ev_kind);
  s->ev_kind = nullptr;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 4D map over one FP32 f buffer: (x, y, z, field) with the padded pitches;
// box = one plane tile with its 2-cell halo, all 15 fields.
bool make_tmap(CUtensorMap* map, void* base, const Layout& L) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)L.sx, (cuuint64_t)(L.ny + 4), (cuuint64_t)(L.nz + 4), (cuuint64_t)lbm::NV};
  const cuuint64_t strides[3] = {(cuuint64_t)L.sx * 4, (cuuint64_t)L.plane * 4, (cuuint64_t)L.fs * 4};
  const cuuint32_t box[4] = {(cuuint32_t)lbm::tiled_box_x(), (cuuint32_t)lbm::tiled_box_y(), 1, (cuuint32_t)lbm::NV};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// z planes per CTA of the tiled kernel: about four waves of two CTAs per SM.
int auto_zchunk(const Layout& L, int num_sms) {
  const long long tiles = (long long)((L.nx + lbm::kTileX - 1) / lbm::kTileX) * ((L.ny + lbm::kTileY - 1) / lbm::kTileY);
  const long long want = 4LL * 2 * num_sms;
  long long chunks = (want + tiles - 1) / tiles;
  long long maxc = L.nz / 8 > 0 ? L.nz / 8 : 1;
  if (chunks > maxc) chunks = maxc;
  if (chunks < 1) chunks = 1;
  return (int)((L.nz + chunks - 1) / chunks);
}

}  // namespace

#define LBM_LAUNCH(sim, kind, expr)                        \
  do {                                                     \
    LBM_CK((sim), begin_launch((sim), (kind)));            \
    LBM_CK((sim), end_launch((sim), (expr)));              \
  } while (0)

extern "C" {

size_t lbm_workspace_bytes(const lbm_grid* grid, int32_t precision) {
  if (!grid_ok(grid) || (precision != LBM_FP64 && precision != LBM_FP32)) return 0;
  const Layout L = make_layout(grid);
  const int esz = precision == LBM_FP64 ? 8 : 4;
  return 2 * field_bytes(L, esz) + kRedBytes + kStatusBytes;
}

int lbm_create(const lbm_grid* grid, const lbm_vset* vset, double tau, double dt, double dx, int32_t precision,
               void* d_workspace, size_t ws_bytes, void* cuda_stream, lbm_sim** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!grid_ok(grid) || !vset || !d_workspace) return LBM_EINVAL;
  if (precision != LBM_FP64 && precision != LBM_FP32) return LBM_EINVAL;
  if (!(std::isfinite(vset->c1) && std::isfinite(vset->c2) && vset->c1 > 0 && vset->c2 > 0 && vset->c1 != vset->c2))
    return LBM_EINVAL;
  if (!(vset->eta0 > 0 && std::isfinite(vset->eta0)) || !(vset->gamma > 1.0 && std::isfinite(vset->gamma)))
    return LBM_EINVAL;
  if (!(tau > 0) || !(dt > 0) || !(dx > 0) || !std::isfinite(dt) || !std::isfinite(dx) || std::isnan(tau))
    return LBM_EINVAL;
  if (((uintptr_t)d_workspace) % kAlign) return LBM_EINVAL;
  const size_t need = lbm_workspace_bytes(grid, precision);
  if (ws_bytes < need) return LBM_ENOMEM;

  lbm_sim* s = new (std::nothrow) lbm_sim();
  if (!s) return LBM_ENOMEM;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return LBM_ECUDA;
  }
  s->prec = precision;
  s->esz = precision == LBM_FP64 ? 8 : 4;
  s->L = make_layout(grid);
  s->vset = *vset;
  s->tau = tau;
  s->dt = dt;
  s->dx = dx;
  s->scheme = LBM_SCHEME_NND;
  s->dissipation = 1;
  s->md = make_model(vset, tau, dt, dx, 1);
  s->mf = to_float(s->md);
  for (int a = 0; a < 3; ++a) {
    s->bc.kind[2 * a] = grid->bc_lo[a];
    s->bc.kind[2 * a + 1] = grid->bc_hi[a];
    for (int k = 0; k < 5; ++k) {
      s->bc.fixed[2 * a][k] = grid->fixed_lo[a][k];
      s->bc.fixed[2 * a + 1][k] = grid->fixed_hi[a][k];
    }
  }
  s->ws = (char*)d_workspace;
  s->ws_bytes = ws_bytes;
  const size_t fb = field_bytes(s->L, s->esz);
  s->fbuf[0] = s->ws;
  s->fbuf[1] = s->ws + fb;
  s->partials = (double*)(s->ws + 2 * fb);
  char* status = s->ws + 2 * fb + kRedBytes;
  s->flags = (unsigned*)status;
  s->counter = (unsigned*)(status + 4);
  s->result = (double*)(status + 64);
  s->cur = 0;
  s->st = (cudaStream_t)cuda_stream;
  s->steps = 0;
  s->failed = 0;
  for (int k = 0; k < LBM_NKERNEL; ++k) {
    s->launches[k] = 0;
    s->ms[k] = 0.0;
  }
  s->variant = LBM_VARIANT_TILED;
  s->zchunk = 0;
  s->num_sms = 0;
  if (cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
      s->num_sms < 1) {
    delete s;
    return LBM_ECUDA;
  }
  if (precision == LBM_FP32) {
    if (!make_tmap(&s->tmap[0], s->fbuf[0], s->L) || !make_tmap(&s->tmap[1], s->fbuf[1], s->L)) {
      delete s;
      return LBM_ECUDA;
    }
  }
  s->timing = 0;
  s->ev = nullptr;
  s->ev_kind = nullptr;
  s->ev_head = s->ev_tail = 0;
  if (cudaMemsetAsync(status, 0, kStatusBytes, s->st) != cudaSuccess) {
    delete s;
    return LBM_ECUDA;
  }
  *out = s;
  return LBM_OK;
}

int lbm_set_scheme(lbm_sim* s, int32_t scheme, int32_t dissipation) {
  if (!s) return LBM_EINVAL;
  if (s->failed) return LBM_ESTATE;
  if (scheme < LBM_SCHEME_NND || scheme > LBM_SCHEME_UPWIND1 || (dissipation != 0 && dissipation != 1))
    return LBM_EINVAL;
  s->scheme = scheme;
  s->dissipation = dissipation;
  s->md = make_model(&s->vset, s->tau, s->dt, s->dx, dissipation);
  s->mf = to_float(s->md);
  return LBM_OK;
}

int lbm_set_launch(lbm_sim* s, int32_t variant, int32_t zchunk) {
  if (!s) return LBM_EINVAL;
  if (s->failed) return LBM_ESTATE;
  if ((variant != LBM_VARIANT_TILED && variant != LBM_VARIANT_PLAIN) || zchunk < 0) return LBM_EINVAL;
  s->variant = variant;
  s->zchunk = zchunk;
  return LBM_OK;
}

int lbm_init(lbm_sim* s, const double* rho, const double* u, const double* T, int32_t on_device) {
  int rc = enter(s);
  if (rc) return rc;
  if (!rho || !u || !T) return LBM_EINVAL;
  const long long n = s->L.ncell();
  s->cur = 0;
  s->steps = 0;
  LBM_CK(s, cudaMemsetAsync(s->flags, 0, sizeof(unsigned), s->st));
  if (on_device) {
    LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_init(s->prec, s->fbuf[0], s->L, s->md, rho, u, T, s->st));
    return LBM_OK;
  }
  double* stg = (double*)s->fbuf[1];
  LBM_CK(s, cudaMemcpyAsync(stg, rho, n * sizeof(double), cudaMemcpyHostToDevice, s->st));
  LBM_CK(s, cudaMemcpyAsync(stg + n, u, 3 * n * sizeof(double), cudaMemcpyHostToDevice, s->st));
  LBM_CK(s, cudaMemcpyAsync(stg + 4 * n, T, n * sizeof(double), cudaMemcpyHostToDevice, s->st));
  LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_init(s->prec, s->fbuf[0], s->L, s->md, stg, stg + n, stg + 4 * n, s->st));
  LBM_CK(s, cudaStreamSynchronize(s->st));
  return LBM_OK;
}

int lbm_step(lbm_sim* s, int64_t n) {
  int rc = enter(s);
  if (rc) return rc;
  if (n < 0) return LBM_EINVAL;
  for (int64_t k = 0; k < n; ++k) {
    void* fin = s->fbuf[s->cur];
    void* fout = s->fbuf[s->cur ^ 1];
    LBM_LAUNCH(s, LBM_KERNEL_FILL, lbm::launch_fill(s->prec, fin, s->L, s->md, s->bc, s->st));
    if (s->prec == LBM_FP32 && s->variant == LBM_VARIANT_TILED) {
      const int zc = s->zchunk > 0 ? s->zchunk : auto_zchunk(s->L, s->num_sms);
      LBM_LAUNCH(s, LBM_KERNEL_STEP,
                 lbm::launch_step_tiled(s->scheme, s->tmap[s->cur], (const float*)fin, (float*)fout, s->L, s->mf, zc,
                                        s->flags, s->st));
    } else {
      LBM_LAUNCH(s, LBM_KERNEL_STEP,
                 lbm::launch_step_plain(s->prec, s->scheme, fin, fout, s->L, s->md, s->mf, s->flags, s->st));
    }
    s->cur ^= 1;
    s->steps += 1;
  }
  return LBM_OK;
}

int lbm_moments(lbm_sim* s, double* rho, double* u, double* T, int32_t on_device) {
  int rc = enter(s);
  if (rc) return rc;
  if (!rho || !u || !T) return LBM_EINVAL;
  const long long n = s->L.ncell();
  if (on_device) {
    LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_moments(s->prec, s->fbuf[s->cur], s->L, s->md, rho, u, T, s->st));
  } else {
    double* stg = (double*)spare(s);
    LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_moments(s->prec, s->fbuf[s->cur], s->L, s->md, stg, stg + n, stg + 4 * n, s->st));
    LBM_CK(s, cudaMemcpyAsync(rho, stg, n * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    LBM_CK(s, cudaMemcpyAsync(u, stg + n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    LBM_CK(s, cudaMemcpyAsync(T, stg + 4 * n, n * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  }
  LBM_CK(s, cudaStreamSynchronize(s->st));
  return LBM_OK;
}

int lbm_get_f(lbm_sim* s, void* f, int32_t on_device) {
  int rc = enter(s);
  if (rc) return rc;
  if (!f) return LBM_EINVAL;
  const size_t bytes = (size_t)lbm::NV * (size_t)s->L.ncell() * s->esz;
  if (on_device) {
    LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_pack(s->prec, s->fbuf[s->cur], s->L, f, s->st));
  } else {
    void* stg = spare(s);
    LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_pack(s->prec, s->fbuf[s->cur], s->L, stg, s->st));
    LBM_CK(s, cudaMemcpyAsync(f, stg, bytes, cudaMemcpyDeviceToHost, s->st));
  }
  LBM_CK(s, cudaStreamSynchronize(s->st));
  return LBM_OK;
}

int lbm_set_f(lbm_sim* s, const void* f, int32_t on_device) {
  int rc = enter(s);
  if (rc) return rc;
  if (!f) return LBM_EINVAL;
  const size_t bytes = (size_t)lbm::NV * (size_t)s->L.ncell() * s->esz;
  s->cur = 0;
  s->steps = 0;
  LBM_CK(s, cudaMemsetAsync(s->flags, 0, sizeof(unsigned), s->st));
  if (on_device) {
    LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_unpack(s->prec, s->fbuf[0], s->L, f, s->st));
    return LBM_OK;
  }
  void* stg = s->fbuf[1];
  LBM_CK(s, cudaMemcpyAsync(stg, f, bytes, cudaMemcpyHostToDevice, s->st));
  LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_unpack(s->prec, s->fbuf[0], s->L, stg, s->st));
  LBM_CK(s, cudaStreamSynchronize(s->st));
  return LBM_OK;
}

int lbm_conserved(lbm_sim* s, double out[5]) {
  int rc = enter(s);
  if (rc) return rc;
  if (!out) return LBM_EINVAL;
  LBM_LAUNCH(s, LBM_KERNEL_REDUCE,
             lbm::launch_conserved(s->prec, s->fbuf[s->cur], s->L, s->md, s->partials, kMaxRedBlocks, s->counter,
                                   s->result, s->flags, s->st));
  unsigned flags = 0;
  LBM_CK(s, cudaMemcpyAsync(out, s->result, 5 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  LBM_CK(s, cudaMemcpyAsync(&flags, s->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st));
  LBM_CK(s, cudaStreamSynchronize(s->st));
  if (flags & LBM_HEALTH_TIMEOUT) return LBM_ETIMEOUT;
  return flags ? LBM_ENONFINITE : LBM_OK;
}

int lbm_health(lbm_sim* s, uint32_t* flags_out) {
  int rc = enter(s);
  if (rc) return rc;
  unsigned flags = 0;
  LBM_CK(s, cudaMemcpyAsync(&flags, s->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st));
  LBM_CK(s, cudaStreamSynchronize(s->st));
  if (flags_out) *flags_out = flags;
  if (flags & LBM_HEALTH_TIMEOUT) return LBM_ETIMEOUT;
  return flags ? LBM_ENONFINITE : LBM_OK;
}

int lbm_sync(lbm_sim* s) {
  int rc = enter(s);
  if (rc) return rc;
  LBM_CK(s, cudaStreamSynchronize(s->st));
  return LBM_OK;
}

int64_t lbm_steps_done(const lbm_sim* s) { return s ? s->steps : -1; }

int lbm_set_timing(lbm_sim* s, int32_t enable) {
  int rc = enter(s);
  if (rc) return rc;
  if (enable && !s->ev) {
    s->ev = (cudaEvent_t*)calloc(2 * kRing, sizeof(cudaEvent_t));
    s->ev_kind = (int*)calloc(kRing, sizeof(int));
    if (!s->ev || !s->ev_kind) {
      free_events(s);
      return LBM_ENOMEM;
    }
    for (int k = 0; k < 2 * kRing; ++k) {
      if (cudaEventCreate(&s->ev[k]) != cudaSuccess) {
        free_events(s);
        return fail(s, cudaErrorMemoryAllocation);
      }
    }
    s->ev_head = s->ev_tail = 0;
  }
  if (!enable && s->ev) {
    while (s->ev_tail < s->ev_head) LBM_CK(s, drain_one(s));
  }
  s->timing = enable ? 1 : 0;
  return LBM_OK;
}

int lbm_get_timing(lbm_sim* s, double* ms, int64_t* launches, int32_t reset) {
  int rc = enter(s);
  if (rc) return rc;
  LBM_CK(s, cudaStreamSynchronize(s->st));
  if (s->ev)
    while (s->ev_tail < s->ev_head) LBM_CK(s, drain_one(s));
  for (int k = 0; k < LBM_NKERNEL; ++k) {
    if (ms) ms[k] = s->ms[k];
    if (launches) launches[k] = s->launches[k];
    if (reset) {
      s->ms[k] = 0.0;
      s->launches[k] = 0;
    }
  }
  return LBM_OK;
}

const char* lbm_status_str(int status) {
  switch (status) {
    case LBM_OK: return "LBM_OK";
    case LBM_EINVAL: return "LBM_EINVAL: invalid argument";
    case LBM_ENOMEM: return "LBM_ENOMEM: workspace too small";
    case LBM_ECUDA: return "LBM_ECUDA: CUDA call failed";
    case LBM_ENONFINITE: return "LBM_ENONFINITE: health flag set (rho<=0, T<=0 or non-finite)";
    case LBM_ETIMEOUT: return "LBM_ETIMEOUT: bounded device wait ran out";
    case LBM_ESTATE: return "LBM_ESTATE: sim failed earlier";
    default: return "unknown lbm status";
  }
}

void lbm_destroy(lbm_sim* s) {
  if (!s) return;
  if (s->ev) {
    cudaStreamSynchronize(s->st);
    free_events(s);
  }
  delete s;
}

}  // extern "C"
