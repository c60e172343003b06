// C ABI of the D3V15 FD-LB solver: argument checks, workspace carving,
// constant tables and kernel sequencing.  Declarations and the contract of
// every entry point are in include/lbm.h.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "lbm_internal.cuh"
#include "tma_ring.cuh"

using lbm::Layout;
using lbm::Model;

namespace {

// NVTX range over one API call (step, batch, graph replay, reduction), for
// profilers that show host-side ranges beside the kernels; a no-op unless a
// tool is attached.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

constexpr size_t kAlign = 256;
constexpr int kMaxRedBlocks = 2048;
constexpr size_t kRedBytes = (size_t)kMaxRedBlocks * 16 * sizeof(double);  // 15 field totals per block
constexpr size_t kStatusBytes = 256;
constexpr double kDefaultKappaMax = 0.0;  // FP64 temperature recovery threshold (0 = off)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool grid_ok(const lbm_grid* g) {
  if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1) return false;
  if (g->nz > 65535 || g->ny > 65535 * 8) return false;
  const int n[3] = {g->nx, g->ny, g->nz};
  for (int a = 0; a < 3; ++a) {
    for (int h = 0; h < 2; ++h) {
      const int k = h ? g->bc_hi[a] : g->bc_lo[a];
      if (k < LBM_BC_PERIODIC || k > LBM_BC_EXTERNAL) return false;
      if ((k == LBM_BC_EXTRAPOLATE || k == LBM_BC_EXTERNAL) && n[a] < 2) return false;
      if (k == LBM_BC_EXTERNAL && a != 0) return false;  // slabs are cut along x
    }
    if ((g->bc_lo[a] == LBM_BC_PERIODIC) != (g->bc_hi[a] == LBM_BC_PERIODIC)) return false;
  }
  // one padded field must hold fewer than 2^32 elements (the tiled kernels
  // index within a field in 32 bits); two FP32 states of that size would
  // already take more than 500 GB
  const size_t sx = align_up((size_t)lbm::OX + (size_t)g->nx + 2, 32);
  const size_t fs = align_up(sx * (size_t)(g->ny + 4) * (size_t)(g->nz + 4), 64);
  return fs <= 0xffffffffull;
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
// FP64 temperature recovery for cells with kappa > kappa_max (0 = off).
lbm::RecoverDesc make_recover(const Model<double>& m, double kappa_max) {
  lbm::RecoverDesc r;
  r.c1 = m.c1;
  r.s = m.s;
  r.eta0sq = m.eta0sq;
  r.c1sq = m.c1sq;
  r.c2sq = m.c2sq;
  r.inv_b = m.inv_b;
  r.axis_w = (float)(6.0 * m.c1sq);
  r.diag_w = (float)(8.0 * m.c2sq);
  r.on = kappa_max > 0.0;
  r.thresh_b = r.on ? (float)((kappa_max - 1.0) / m.inv_b) : 0.0f;
  return r;
}

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
  m.keep0 = 1.0 - m.dt_tau - 6.0 * m.lam0;
  m.keep1 = 1.0 - m.dt_tau - 6.0 * m.lam1;
  m.keep2 = 1.0 - m.dt_tau;
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
  f.keep0 = (float)d.keep0; f.keep1 = (float)d.keep1; f.keep2 = (float)d.keep2;
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
  unsigned long long* queue;  // batched-step work queue (status block)
  unsigned* done;
  double* result;
  cudaStream_t st;
  int64_t steps;
  int failed;
  unsigned external;    // faces (bit 2*axis+hi) whose layers the caller supplies (LBM_BC_EXTERNAL)
  unsigned halo_set;    // EXTERNAL faces written by lbm_set_halo since the last step
  int fixed_dirty[2];   // FIXED-face layers of buffer b need rewriting
  int layers_ok[2];     // buffer b's non-FIXED boundary layers match its interior
  unsigned wait_limit;  // polls of a TMA data wait before the step kernel gives up
  int variant;          // LBM_VARIANT_* of the FP32 step
  int zchunk;           // z planes per unit of the tiled kernels, 0 = automatic
  int ztail;            // pair kernels: short chunks of ztail planes end the z range (0 = none)
  int num_sms;
  CUtensorMap tmap[2];  // FP32: TMA descriptors of the two f buffers, box 40 x 12 x 1 x 15 (32 x 8 tiles)
  CUtensorMap wmap[2];  // the same with box 72 x 12 x 1 x 15 (64 x 8 tiles, variant TILED64)
  lbm::RecoverDesc rd;  // FP64 temperature recovery of the pair kernel
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

// The buffer not holding the current state; host-pointer transfers stage
// through it, which overwrites its boundary layers.
void* spare(lbm_sim* s) {
  s->fixed_dirty[s->cur ^ 1] = 1;
  s->layers_ok[s->cur ^ 1] = 0;
  return s->fbuf[s->cur ^ 1];
}

// Faces whose layers change from step to step (all but FIXED), and the FIXED
// ones, whose layers are written once per buffer when the state is set.
unsigned step_faces(const lbm_sim* s);
unsigned fixed_faces(const lbm_sim* s);

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
// box = one plane tile with its 2-cell halo (bx x by), all 15 fields.
bool make_tmap(CUtensorMap* map, void* base, const Layout& L, int bx, int by) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)L.sx, (cuuint64_t)(L.ny + 4), (cuuint64_t)(L.nz + 4), (cuuint64_t)lbm::NV};
  const cuuint64_t strides[3] = {(cuuint64_t)L.sx * 4, (cuuint64_t)L.plane * 4, (cuuint64_t)L.fs * 4};
  const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, (cuuint32_t)lbm::NV};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, lbm::ring::kPlaneL2Promotion,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Variants whose step kernel writes the boundary layers of its output.
bool wt_variant(int variant) {
  return variant == LBM_VARIANT_TILED || variant == LBM_VARIANT_TILED64 || variant == LBM_VARIANT_TILED_SPLIT;
}

// Variants that run the pair kernel, and its tile width.
bool pair_variant(int variant) {
  return variant == LBM_VARIANT_TILED || variant == LBM_VARIANT_TILED_FILL || variant == LBM_VARIANT_TILED64 ||
         variant == LBM_VARIANT_TILED_SPLIT;
}
int pair_cols(int variant) { return variant == LBM_VARIANT_TILED64 ? 64 : 32; }

// z planes per CTA of the tiled kernels (`cols` x 8 tiles, `ctas` CTAs per
// SM) when none is set: the largest of 32, 24, 16, 12, 8, 6, 4 that still
// gives two waves of units.  Each unit re-reads four planes around its chunk
// and pays a prologue, so long chunks save work; short chunks fill the SMs.
// The pair kernels then end each column in 8-plane chunks (auto_ztail), so
// the last wave is short.  Measured on GB300 (32 x 8 tiles): 256^3 gets 32 + 8
// (0.464-0.469 ms; equal 16 / 24 / 32: 0.481 / 0.472 / 0.482), 192^3 32 + 8
// (0.218; best measured 0.216), 128^3 12 + 8 (equal 12: 0.085).  The
// autotuner (autotune.py) measures the choice per grid.
int auto_zchunk(const Layout& L, int num_sms, int cols, int ctas) {
  const long long tiles = (long long)((L.nx + cols - 1) / cols) * ((L.ny + lbm::kTileY - 1) / lbm::kTileY);
  const long long want = 2LL * ctas * num_sms;
  static const int cand[] = {32, 24, 16, 12, 8, 6, 4};
  for (int zc : cand)
    if (tiles * ((L.nz + zc - 1) / zc) >= want) return zc < L.nz ? zc : L.nz;
  return L.nz < 4 ? L.nz : 4;
}
int auto_ztail(int zc) { return zc >= 12 ? 8 : 0; }

unsigned step_faces(const lbm_sim* s) {
  unsigned m = 0;
  for (int f = 0; f < 6; ++f)
    if (s->bc.kind[f] != LBM_BC_FIXED && s->bc.kind[f] != LBM_BC_EXTERNAL) m |= 1u << f;
  return m;
}

unsigned fixed_faces(const lbm_sim* s) {
  unsigned m = 0;
  for (int f = 0; f < 6; ++f)
    if (s->bc.kind[f] == LBM_BC_FIXED) m |= 1u << f;
  return m;
}

// Boundary layers the pair kernel writes for the state it produces, and the
// face mask they cover: periodic axes (x only for even nx, where the boundary
// cell pairs are whole) and extrapolating / reflecting x faces (even nx).
lbm::WtDesc write_through(const lbm_sim* s, unsigned* faces) {
  lbm::WtDesc w;
  unsigned m = 0;
  const bool on = wt_variant(s->variant);
  const bool xeven = (s->L.nx % 2) == 0 && s->L.nx >= 4;
  const int n[3] = {s->L.nx, s->L.ny, s->L.nz};
  for (int a = 0; a < 3; ++a) {
    w.per[a] = on && s->bc.kind[2 * a] == LBM_BC_PERIODIC && n[a] >= 4 && (a != 0 || xeven);
    if (w.per[a]) m |= 3u << (2 * a);
  }
  auto xk = [&](int kind) {
    return (on && xeven && (kind == LBM_BC_EXTRAPOLATE || kind == LBM_BC_REFLECT)) ? kind : 0;
  };
  w.xlo = xk(s->bc.kind[0]);
  w.xhi = xk(s->bc.kind[1]);
  if (w.xlo) m |= 1u;
  if (w.xhi) m |= 2u;
  if (faces) *faces = m;
  return w;
}

}  // namespace

#define LBM_LAUNCH(sim, kind, expr)                        \
  do {                                                     \
    LBM_CK((sim), begin_launch((sim), (kind)));            \
    LBM_CK((sim), end_launch((sim), (expr)));              \
  } while (0)

namespace {

// FIXED faces hold constant layers: they are written into a buffer once and
// again only after that buffer served as host staging (which overwrites it).
int fill_fixed(lbm_sim* s) {
  const unsigned m = fixed_faces(s);
  for (int b = 0; b < 2; ++b) {
    if (!s->fixed_dirty[b]) continue;
    if (m)
      LBM_LAUNCH(s, LBM_KERNEL_FILL, lbm::launch_fill(s->prec, s->fbuf[b], s->L, s->md, s->mf, s->bc, m, s->st));
    s->fixed_dirty[b] = 0;
  }
  return LBM_OK;
}

}  // namespace

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
  s->rd = make_recover(s->md, kDefaultKappaMax);
  for (int a = 0; a < 3; ++a) {
    s->bc.kind[2 * a] = grid->bc_lo[a];
    s->bc.kind[2 * a + 1] = grid->bc_hi[a];
    for (int k = 0; k < 5; ++k) {
      s->bc.fixed[2 * a][k] = grid->fixed_lo[a][k];
      s->bc.fixed[2 * a + 1][k] = grid->fixed_hi[a][k];
    }
  }
  s->external = 0;
  for (int f = 0; f < 6; ++f)
    if (s->bc.kind[f] == LBM_BC_EXTERNAL) s->external |= 1u << f;
  s->halo_set = 0;
  s->ws = (char*)d_workspace;
  s->ws_bytes = ws_bytes;
  const size_t fb = field_bytes(s->L, s->esz);
  s->fbuf[0] = s->ws;
  s->fbuf[1] = s->ws + fb;
  s->partials = (double*)(s->ws + 2 * fb);
  char* status = s->ws + 2 * fb + kRedBytes;
  s->flags = (unsigned*)status;
  s->counter = (unsigned*)(status + 4);
  s->queue = (unsigned long long*)(status + 16);
  s->done = (unsigned*)(status + 24);
  s->result = (double*)(status + 64);
  s->cur = 0;
  s->st = (cudaStream_t)cuda_stream;
  s->steps = 0;
  s->failed = 0;
  for (int k = 0; k < LBM_NKERNEL; ++k) {
    s->launches[k] = 0;
    s->ms[k] = 0.0;
  }
  s->fixed_dirty[0] = s->fixed_dirty[1] = 1;
  s->layers_ok[0] = s->layers_ok[1] = 0;
  s->variant = LBM_VARIANT_TILED;
  s->wait_limit = 1u << 22;
  s->zchunk = 0;
  s->ztail = 0;
  s->num_sms = 0;
  if (cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
      s->num_sms < 1) {
    delete s;
    return LBM_ECUDA;
  }
  if (precision == LBM_FP32) {
    const lbm::PairShape p64 = lbm::pair_shape(64);
    if (!make_tmap(&s->tmap[0], s->fbuf[0], s->L, lbm::tiled_box_x(), lbm::tiled_box_y()) ||
        !make_tmap(&s->tmap[1], s->fbuf[1], s->L, lbm::tiled_box_x(), lbm::tiled_box_y()) ||
        !make_tmap(&s->wmap[0], s->fbuf[0], s->L, p64.bx, p64.by) ||
        !make_tmap(&s->wmap[1], s->fbuf[1], s->L, p64.bx, p64.by) ||
        lbm::prepare_tiled_kernels() != cudaSuccess || lbm::prepare_pair_kernels() != cudaSuccess ||
        lbm::prepare_split_kernels() != cudaSuccess) {
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

int lbm_set_launch(lbm_sim* s, int32_t variant, int32_t zchunk, int32_t ztail) {
  if (!s) return LBM_EINVAL;
  if (s->failed) return LBM_ESTATE;
  if (variant < LBM_VARIANT_TILED || variant > LBM_VARIANT_TILED_SPLIT || zchunk < 0 || ztail < 0) return LBM_EINVAL;
  s->variant = variant;
  s->zchunk = zchunk;
  s->ztail = ztail;
  s->layers_ok[0] = s->layers_ok[1] = 0;
  return LBM_OK;
}

int lbm_set_t_recovery(lbm_sim* s, double kappa_max) {
  if (!s) return LBM_EINVAL;
  if (s->failed) return LBM_ESTATE;
  if (!(kappa_max == 0.0 || kappa_max >= 1.0)) return LBM_EINVAL;
  s->rd = make_recover(s->md, kappa_max);
  return LBM_OK;
}

int lbm_set_wait_limit(lbm_sim* s, uint32_t polls) {
  if (!s) return LBM_EINVAL;
  if (s->failed) return LBM_ESTATE;
  s->wait_limit = polls;
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
  s->fixed_dirty[0] = s->fixed_dirty[1] = 1;
  s->layers_ok[0] = s->layers_ok[1] = 0;
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

}  // extern "C"

namespace {

// n time steps of one sim (fills as needed, then the step kernel).
int run_steps(lbm_sim* s, int64_t n) {
  if (n > 0) {
    int rc = fill_fixed(s);
    if (rc) return rc;
  }
  const bool pair = s->prec == LBM_FP32 && pair_variant(s->variant);
  const lbm::PairShape shape = lbm::pair_shape(pair_cols(s->variant));
  unsigned wt_faces = 0;
  const lbm::WtDesc wt = write_through(s, &wt_faces);
  for (int64_t k = 0; k < n; ++k) {
    void* fin = s->fbuf[s->cur];
    void* fout = s->fbuf[s->cur ^ 1];
    // layers the previous step did not write for this state
    unsigned mask = step_faces(s);
    if (pair && s->layers_ok[s->cur]) mask &= ~wt_faces;
    if (mask)
      LBM_LAUNCH(s, LBM_KERNEL_FILL, lbm::launch_fill(s->prec, fin, s->L, s->md, s->mf, s->bc, mask, s->st));
    if (s->prec == LBM_FP32 && s->variant != LBM_VARIANT_PLAIN) {
      const int zc = s->zchunk > 0 ? s->zchunk
                                   : (pair ? auto_zchunk(s->L, s->num_sms, shape.tx, shape.ctas_per_sm)
                                           : auto_zchunk(s->L, s->num_sms, lbm::kTileX, 2));
      if (pair) {
        const CUtensorMap& map = shape.tx == 64 ? s->wmap[s->cur] : s->tmap[s->cur];
        const lbm::ZSched zs = lbm::make_zsched(s->L.nz, zc, s->zchunk > 0 ? s->ztail : auto_ztail(zc));
        if (s->variant == LBM_VARIANT_TILED_SPLIT)
          LBM_LAUNCH(s, LBM_KERNEL_STEP,
                     lbm::launch_step_split(s->scheme, map, (const float*)fin, (float*)fout, s->L, s->mf, wt, s->rd, zs,
                                            s->flags, s->wait_limit, s->st));
        else
          LBM_LAUNCH(s, LBM_KERNEL_STEP,
                     lbm::launch_step_pair(shape.tx, s->scheme, map, (const float*)fin, (float*)fout, s->L, s->mf,
                                           wt, s->rd, zs, s->flags, s->wait_limit, s->st));
      } else {
        LBM_LAUNCH(s, LBM_KERNEL_STEP,
                   lbm::launch_step_tiled(s->scheme, s->tmap[s->cur], (const float*)fin, (float*)fout, s->L, s->mf,
                                          zc, s->flags, s->st));
      }
    } else {
      LBM_LAUNCH(s, LBM_KERNEL_STEP,
                 lbm::launch_step_plain(s->prec, s->scheme, fin, fout, s->L, s->md, s->mf, s->flags, s->st));
    }
    s->layers_ok[s->cur ^ 1] = (pair && wt_faces) ? 1 : 0;
    s->cur ^= 1;
    s->steps += 1;
  }
  return LBM_OK;
}

// z planes per unit of the batched kernel when a sim has none set.  Measured
// (GB300): eight 128^3 grids 0.526 / 0.522 / 0.529 ms per step at 16 / 24 / 32
// planes; with the 512 x 256 x 256 grid added 1.430 / 1.394 / 1.386 ms.
constexpr int kBatchZchunk = 24;

int batch_check(lbm_sim* const* sims, int32_t n) {
  if (!sims || n < 1 || n > lbm::kMaxBatch) return LBM_EINVAL;
  for (int i = 0; i < n; ++i) {
    lbm_sim* s = sims[i];
    if (!s) return LBM_EINVAL;
    if (s->failed) return LBM_ESTATE;
    if (s->prec != LBM_FP32 || !wt_variant(s->variant) || s->variant != sims[0]->variant) return LBM_EINVAL;
    if (s->external) return LBM_EINVAL;  // slab sims step one at a time between halo exchanges
    if (s->scheme != sims[0]->scheme || s->st != sims[0]->st || s->device != sims[0]->device) return LBM_EINVAL;
    for (int j = 0; j < i; ++j)
      if (sims[j] == s) return LBM_EINVAL;
  }
  return LBM_OK;
}

// n batched time steps: per-sim fills where needed, then one table-driven
// launch of the persistent tile kernel for all sims.
int run_batch(lbm_sim* const* sims, int32_t n, int64_t steps) {
  lbm_sim* s0 = sims[0];
  const lbm::PairShape shape = lbm::pair_shape(pair_cols(s0->variant));
  for (int i = 0; i < n; ++i) {
    int rc = fill_fixed(sims[i]);
    if (rc) return rc;
  }
  thread_local static lbm::BatchTable tab;  // built on the host, passed by value to the kernel
  unsigned wt_faces[lbm::kMaxBatch];
  lbm::WtDesc wt[lbm::kMaxBatch];
  for (int i = 0; i < n; ++i) wt[i] = write_through(sims[i], &wt_faces[i]);
  for (int64_t k = 0; k < steps; ++k) {
    long long units = 0;
    for (int i = 0; i < n; ++i) {
      lbm_sim* s = sims[i];
      unsigned mask = step_faces(s);
      if (s->layers_ok[s->cur]) mask &= ~wt_faces[i];
      if (mask)
        LBM_LAUNCH(s, LBM_KERNEL_FILL,
                   lbm::launch_fill(s->prec, s->fbuf[s->cur], s->L, s->md, s->mf, s->bc, mask, s->st));
      lbm::BatchItem& it = tab.item[i];
      tab.map[i] = shape.tx == 64 ? s->wmap[s->cur] : s->tmap[s->cur];
      it.fin = (const float*)s->fbuf[s->cur];
      it.fout = (float*)s->fbuf[s->cur ^ 1];
      it.flags = s->flags;
      it.L = s->L;
      it.m = s->mf;
      it.wt = wt[i];
      it.rd = s->rd;
      it.tiles_x = (s->L.nx + shape.tx - 1) / shape.tx;
      it.tiles_y = (s->L.ny + shape.ty - 1) / shape.ty;
      it.zs = s->zchunk > 0 ? lbm::make_zsched(s->L.nz, s->zchunk, s->ztail)
                            : lbm::make_zsched(s->L.nz, kBatchZchunk, 0);
      it.first_unit = units;
      units += (long long)it.tiles_x * it.tiles_y * it.zs.nch;
    }
    tab.n = n;
    tab.wait_limit = s0->wait_limit;
    tab.total_units = units;
    tab.queue = s0->queue;
    tab.done = s0->done;
    const long long resident = (long long)shape.ctas_per_sm * s0->num_sms;
    const int grid = (int)(units < resident ? units : resident);
    if (s0->variant == LBM_VARIANT_TILED_SPLIT)
      LBM_LAUNCH(s0, LBM_KERNEL_STEP, lbm::launch_step_split_batch(s0->scheme, tab, grid, s0->st));
    else
      LBM_LAUNCH(s0, LBM_KERNEL_STEP, lbm::launch_step_pair_batch(shape.tx, s0->scheme, tab, grid, s0->st));
    for (int i = 0; i < n; ++i) {
      lbm_sim* s = sims[i];
      s->layers_ok[s->cur ^ 1] = 1;
      s->cur ^= 1;
      s->steps += 1;
    }
  }
  return LBM_OK;
}

}  // namespace

struct lbm_graph {
  cudaGraphExec_t exec;
  cudaStream_t st;
  int n;
  lbm_sim* sims[lbm::kMaxBatch];
  int cur[lbm::kMaxBatch];
  int64_t steps;
  int64_t launches[LBM_NKERNEL];  // per replay, booked on sims[0]
};

extern "C" {

int lbm_step(lbm_sim* s, int64_t n) {
  Range r("lbm_step");
  int rc = enter(s);
  if (rc) return rc;
  if (n < 0) return LBM_EINVAL;
  if (s->external && n > 0) {
    // the caller's layers are one step's worth: one step at a time, each after its lbm_set_halo calls
    if (n != 1 || (s->halo_set & s->external) != s->external) return LBM_EINVAL;
    s->halo_set = 0;
  }
  return run_steps(s, n);
}

int lbm_get_halo_source(lbm_sim* s, int32_t side, void* buf, int32_t on_device) {
  int rc = enter(s);
  if (rc) return rc;
  if (!buf || (side != 0 && side != 1) || s->L.nx < 2) return LBM_EINVAL;
  const size_t bytes = (size_t)lbm::NV * s->L.ny * s->L.nz * 2 * s->esz;
  if (on_device) {
    LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_halo(s->prec, s->fbuf[s->cur], s->L, side, 1, buf, s->st));
    return LBM_OK;
  }
  void* stg = spare(s);
  LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_halo(s->prec, s->fbuf[s->cur], s->L, side, 1, stg, s->st));
  LBM_CK(s, cudaMemcpyAsync(buf, stg, bytes, cudaMemcpyDeviceToHost, s->st));
  LBM_CK(s, cudaStreamSynchronize(s->st));
  return LBM_OK;
}

int lbm_set_halo(lbm_sim* s, int32_t side, const void* buf, int32_t on_device) {
  int rc = enter(s);
  if (rc) return rc;
  if (!buf || (side != 0 && side != 1) || !((s->external >> side) & 1u)) return LBM_EINVAL;
  const size_t bytes = (size_t)lbm::NV * s->L.ny * s->L.nz * 2 * s->esz;
  if (on_device) {
    LBM_LAUNCH(s, LBM_KERNEL_OTHER,
               lbm::launch_halo(s->prec, s->fbuf[s->cur], s->L, side, 0, const_cast<void*>(buf), s->st));
  } else {
    void* stg = spare(s);
    LBM_CK(s, cudaMemcpyAsync(stg, buf, bytes, cudaMemcpyHostToDevice, s->st));
    LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_halo(s->prec, s->fbuf[s->cur], s->L, side, 0, stg, s->st));
    LBM_CK(s, cudaStreamSynchronize(s->st));
  }
  s->halo_set |= 1u << side;
  return LBM_OK;
}

int lbm_step_batch(lbm_sim* const* sims, int32_t n, int64_t steps) {
  Range r("lbm_step_batch");
  int rc = batch_check(sims, n);
  if (rc) return rc;
  rc = enter(sims[0]);
  if (rc) return rc;
  if (steps < 0) return LBM_EINVAL;
  return run_batch(sims, n, steps);
}

int lbm_graph_capture(lbm_sim* const* sims, int32_t n, int64_t steps, lbm_graph** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!sims || n < 1 || steps < 2 || steps % 2) return LBM_EINVAL;
  int rc = n == 1 ? (sims[0] ? (sims[0]->external ? LBM_EINVAL : LBM_OK) : LBM_EINVAL) : batch_check(sims, n);
  if (rc) return rc;
  lbm_sim* s0 = sims[0];
  rc = enter(s0);
  if (rc) return rc;
  // boundary layers that only need writing once are written now, outside the graph
  for (int i = 0; i < n; ++i) {
    lbm_sim* s = sims[i];
    rc = fill_fixed(s);
    if (rc) return rc;
    if (!s->layers_ok[s->cur]) {
      const unsigned mask = step_faces(s);
      if (mask)
        LBM_LAUNCH(s, LBM_KERNEL_FILL, lbm::launch_fill(s->prec, s->fbuf[s->cur], s->L, s->md, s->mf, s->bc, mask,
                                                        s->st));
      s->layers_ok[s->cur] = s->prec == LBM_FP32 && wt_variant(s->variant);
    }
  }
  lbm_graph* g = new (std::nothrow) lbm_graph();
  if (!g) return LBM_ENOMEM;
  g->st = s0->st;
  g->n = n;
  g->steps = steps;
  // the capture records launches without running them: save the host-side
  // state it advances and restore it afterwards
  int64_t saved_steps[lbm::kMaxBatch], saved_launch[lbm::kMaxBatch][LBM_NKERNEL];
  int saved_timing[lbm::kMaxBatch], saved_ok[lbm::kMaxBatch][2];
  for (int i = 0; i < n; ++i) {
    lbm_sim* s = sims[i];
    g->sims[i] = s;
    g->cur[i] = s->cur;
    saved_steps[i] = s->steps;
    saved_timing[i] = s->timing;
    saved_ok[i][0] = s->layers_ok[0];
    saved_ok[i][1] = s->layers_ok[1];
    for (int k = 0; k < LBM_NKERNEL; ++k) saved_launch[i][k] = s->launches[k];
    s->timing = 0;
  }
  // capture on a private stream (the sims' stream may be the legacy default
  // stream, which cannot be captured); replays run on the sims' stream
  cudaGraph_t graph = nullptr;
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    for (int i = 0; i < n; ++i) sims[i]->st = cap;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = n == 1 ? run_steps(s0, steps) : run_batch(sims, n, steps);
      cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
      if (e == cudaSuccess) e = e2;
    }
    for (int i = 0; i < n; ++i) sims[i]->st = g->st;
    cudaStreamDestroy(cap);
  }
  for (int k = 0; k < LBM_NKERNEL; ++k) g->launches[k] = s0->launches[k] - saved_launch[0][k];
  if (n > 1)
    for (int i = 1; i < n; ++i)
      for (int k = 0; k < LBM_NKERNEL; ++k) g->launches[k] += sims[i]->launches[k] - saved_launch[i][k];
  for (int i = 0; i < n; ++i) {
    lbm_sim* s = sims[i];
    s->steps = saved_steps[i];
    s->timing = saved_timing[i];
    s->cur = g->cur[i];
    s->layers_ok[0] = saved_ok[i][0];
    s->layers_ok[1] = saved_ok[i][1];
    for (int k = 0; k < LBM_NKERNEL; ++k) s->launches[k] = saved_launch[i][k];
  }
  if (e == cudaSuccess && rc == LBM_OK) e = cudaGraphInstantiate(&g->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (rc != LBM_OK || e != cudaSuccess) {
    delete g;
    if (rc != LBM_OK) return rc;
    for (int i = 0; i < n; ++i) sims[i]->failed = 1;
    return LBM_ECUDA;
  }
  *out = g;
  return LBM_OK;
}

int lbm_graph_launch(lbm_graph* g) {
  Range r("lbm_graph_launch");
  if (!g) return LBM_EINVAL;
  for (int i = 0; i < g->n; ++i) {
    if (g->sims[i]->failed) return LBM_ESTATE;
    if (g->sims[i]->cur != g->cur[i]) return LBM_ESTATE;
  }
  lbm_sim* s0 = g->sims[0];
  int rc = enter(s0);
  if (rc) return rc;
  LBM_CK(s0, cudaGraphLaunch(g->exec, g->st));
  for (int i = 0; i < g->n; ++i) {
    lbm_sim* s = g->sims[i];
    s->steps += g->steps;
    if (s->prec == LBM_FP32 && wt_variant(s->variant)) s->layers_ok[s->cur] = 1;
  }
  for (int k = 0; k < LBM_NKERNEL; ++k) s0->launches[k] += g->launches[k];
  return LBM_OK;
}

void lbm_graph_destroy(lbm_graph* g) {
  if (!g) return;
  cudaStreamSynchronize(g->st);
  cudaGraphExecDestroy(g->exec);
  delete g;
}

}  // extern "C"

extern "C" {

int lbm_moments(lbm_sim* s, double* rho, double* u, double* T, int32_t on_device) {
  int rc = enter(s);
  if (rc) return rc;
  if (!rho || !u || !T) return LBM_EINVAL;
  const long long n = s->L.ncell();
  if (on_device) {
    LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_moments(s->prec, s->fbuf[s->cur], s->L, s->md, rho, u, T, s->st));
  } else {
    double* stg = (double*)spare(s);
    LBM_LAUNCH(s, LBM_KERNEL_OTHER,
               lbm::launch_moments(s->prec, s->fbuf[s->cur], s->L, s->md, stg, stg + n, stg + 4 * n, s->st));
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
  s->fixed_dirty[0] = s->fixed_dirty[1] = 1;
  s->layers_ok[0] = s->layers_ok[1] = 0;
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
  Range r("lbm_conserved");
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

int lbm_moments_async(lbm_sim* s, double* rho, double* u, double* T) {
  int rc = enter(s);
  if (rc) return rc;
  if (!rho || !u || !T) return LBM_EINVAL;
  LBM_LAUNCH(s, LBM_KERNEL_OTHER, lbm::launch_moments(s->prec, s->fbuf[s->cur], s->L, s->md, rho, u, T, s->st));
  return LBM_OK;
}

int lbm_health_async(lbm_sim* s, uint32_t* flags_out) {
  int rc = enter(s);
  if (rc) return rc;
  if (!flags_out) return LBM_EINVAL;
  LBM_CK(s, cudaMemcpyAsync(flags_out, s->flags, sizeof(unsigned), cudaMemcpyDefault, s->st));
  return LBM_OK;
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

extern "C" int lbm_vn_max_growth(const double* states, int32_t nstates, const double* params, int32_t nparams,
                                 const double* dirs, int32_t ndirs, int32_t nk, int32_t dissipation, double* out,
                                 void* cuda_stream) {
  if (!states || !params || !dirs || !out || nstates < 1 || nparams < 1 || ndirs < 1 || nk < 1) return LBM_EINVAL;
  const long long items = (long long)nstates * ndirs * nk * nparams;
  if (items > (1LL << 30)) return LBM_EINVAL;
  return lbm::launch_vn_max_growth(states, nstates, params, nparams, dirs, ndirs, nk, dissipation, out,
                                   (cudaStream_t)cuda_stream) == cudaSuccess
             ? LBM_OK
             : LBM_ECUDA;
}

extern "C" int lbm_reciprocal_fp32(const float* x, float* y, int64_t n, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return LBM_EINVAL;
  return lbm::launch_reciprocal_fp32(x, y, (long long)n, (cudaStream_t)cuda_stream) == cudaSuccess ? LBM_OK
                                                                                                    : LBM_ECUDA;
}
