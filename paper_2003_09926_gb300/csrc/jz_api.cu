// jz_api.cu -- host side of the C ABI declared in include/jz.h: descriptor
// validation, carving of the caller's device buffer, the per-step launch
// sequence, CUDA-graph replay, diagnostics and host<->device state copies.
//
// Per time step (arXiv 2003.09926, Section 4.2, Fig. jazzy; the ghost
// exchanges of the paper become the boundary fill of the two-layer fringe):
//   time step (CFL reduction or fixed dt)
//   stage 1: Q0 -> QA     [boundary fill of QA]
//   stage 2: QA -> QB     [boundary fill of QB]
//   stage 3: QB -> QA     [boundary fill of QA]
//   stage 4: QA -> QB     [boundary fill of QB]
//   stage 5: QB -> Q0 (in place: each node reads its own Q0 before writing)
//   boundary fill of Q0
// Stage 1 needs no boundary fill: Q^n already carries its boundary values,
// which depend only on interior nodes.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "jz_internal.h"

namespace jz {

static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static thread_local std::string g_error;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
  return code;
}

int record_error(int code, const char* msg) { return fail(code, "%s", msg); }

#define JZ_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(JZ_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carve {
  Layout L;
  size_t es, ms;  // state / metric element sizes
  size_t off_sc, off_partial, off_tab, off_inflow, off_axis, off_q0, off_qa, off_qb, off_m, off_q0d, total;
  size_t tab_len;
};

static int validate(const jz_grid_desc* d) {
  if (!d) return fail(JZ_EINVAL, "null descriptor");
  int n[3] = {d->ni, d->nj, d->nk};
  for (int a = 0; a < 3; ++a) {
    int b0 = d->bc[2 * a], b1 = d->bc[2 * a + 1];
    for (int b : {b0, b1})
      if (b != JZ_BC_PERIODIC && b != JZ_BC_INFLOW && b != JZ_BC_FARFIELD && b != JZ_BC_AXIS)
        return fail(JZ_EINVAL, "bad boundary kind %d", b);
    if ((b0 == JZ_BC_PERIODIC) != (b1 == JZ_BC_PERIODIC))
      return fail(JZ_EINVAL, "direction %d: both faces or neither must be periodic", a);
    bool per = b0 == JZ_BC_PERIODIC;
    if (per ? n[a] < 1 : n[a] < 3) return fail(JZ_EINVAL, "direction %d: %d nodes is too few", a, n[a]);
    if (n[a] > (1 << 24)) return fail(JZ_EINVAL, "direction %d: %d nodes is too many", a, n[a]);
    if (!(d->hi[a] > d->lo[a])) return fail(JZ_EINVAL, "direction %d: empty extent", a);
  }
  for (int f = 1; f < 6; ++f)
    if (d->bc[f] == JZ_BC_INFLOW) return fail(JZ_EINVAL, "the inflow condition is supported on the x- face only");
  if ((long long)d->nj * d->nk * ((d->ni + 31) / 32) >= (1LL << 31))
    return fail(JZ_EINVAL, "grid too large: nj * nk * ceil(ni / 32) must stay below 2^31");
  if (d->precision != JZ_P64 && d->precision != JZ_P32_M64 && d->precision != JZ_P32 && d->precision != JZ_P32_S64)
    return fail(JZ_EINVAL, "bad precision mode %d", d->precision);
  if (d->stretch_c != 0.0 && !(d->stretch_w > 0.0)) return fail(JZ_EINVAL, "stretch_w must be > 0");
  if (!std::isfinite(d->map_amp) || !std::isfinite(d->stretch_c) || !std::isfinite(d->cluster_r))
    return fail(JZ_EINVAL, "non-finite grid parameter");
  if (d->geom != JZ_GEOM_BOX && d->geom != JZ_GEOM_CYLINDER) return fail(JZ_EINVAL, "bad geometry %d", d->geom);
  for (int f = 0; f < 6; ++f)
    if (d->bc[f] == JZ_BC_AXIS && !(f == 2 && d->geom == JZ_GEOM_CYLINDER))
      return fail(JZ_EINVAL, "the centreline condition is the y- face of a cylindrical grid only");
  if (d->geom == JZ_GEOM_CYLINDER) {
    if (d->bc[2] != JZ_BC_AXIS) return fail(JZ_EINVAL, "a cylindrical grid needs JZ_BC_AXIS on its y- face");
    if (d->bc[4] != JZ_BC_PERIODIC) return fail(JZ_EINVAL, "a cylindrical grid is periodic in k");
    if (d->bc[0] == JZ_BC_PERIODIC || d->bc[3] == JZ_BC_PERIODIC)
      return fail(JZ_EINVAL, "a cylindrical grid is not periodic in i or j");
    if (d->nk < 5 || (d->nk - 1) % 2 != 0)
      return fail(JZ_EINVAL, "a cylindrical grid needs nk - 1 even and nk >= 5 (got %d)", d->nk);
    if (d->nj < 4) return fail(JZ_EINVAL, "a cylindrical grid needs nj >= 4");
    if (d->lo[1] != 0.0) return fail(JZ_EINVAL, "a cylindrical grid's radius starts at lo[1] = 0");
    if (d->map_amp != 0.0) return fail(JZ_EINVAL, "a cylindrical grid takes no sinusoidal mapping");
  }
  return JZ_OK;
}

// Nodes [o0, o1] of the grid d (the whole grid when o0 is null): a face of
// the block that lies inside the grid is an exchange face, whose first /
// last node is updated and whose ghosts are filled by the halo exchange.
// Block [o0, o1] of the grid d: inside the grid, not split across a periodic
// direction, and at least three nodes deep along a split direction (its
// neighbours copy two layers of its nodes into their ghosts)
static int validate_block(const jz_grid_desc* d, const int* o0, const int* o1) {
  if (!o0 || !o1) return fail(JZ_EINVAL, "null block range");
  const int gn[3] = {d->ni, d->nj, d->nk};
  for (int a = 0; a < 3; ++a) {
    if (o0[a] < 0 || o1[a] > gn[a] - 1 || o1[a] < o0[a])
      return fail(JZ_EINVAL, "direction %d: block range [%d, %d] outside the grid's [0, %d]", a, o0[a], o1[a],
                  gn[a] - 1);
    const bool split = o0[a] > 0 || o1[a] < gn[a] - 1;
    if (split && d->bc[2 * a] == JZ_BC_PERIODIC) return fail(JZ_EINVAL, "direction %d: a periodic direction cannot be split", a);
    if (split && a > 0 && d->geom == JZ_GEOM_CYLINDER)
      return fail(JZ_EINVAL, "direction %d: a cylindrical grid may be split in i only", a);
    if (split && o1[a] - o0[a] + 1 < 3)
      return fail(JZ_EINVAL, "direction %d: a block of a split direction needs at least 3 nodes", a);
  }
  return JZ_OK;
}

static Carve carve(const jz_grid_desc* d, const int* o0 = nullptr, const int* o1 = nullptr) {
  Carve c;
  Layout& L = c.L;
  const int gn[3] = {d->ni, d->nj, d->nk};
  for (int a = 0; a < 3; ++a) {
    const int b0 = o0 ? o0[a] : 0, b1 = o1 ? o1[a] : gn[a] - 1;
    L.n[a] = b1 - b0 + 1;
    L.per[a] = d->bc[2 * a] == JZ_BC_PERIODIC;
    // azimuth of a cylinder: the last node repeats the first
    L.pn[a] = (d->geom == JZ_GEOM_CYLINDER && a == 2) ? L.n[a] - 1 : L.n[a];
    L.bc[2 * a] = b0 > 0 ? BC_EXCHANGE : d->bc[2 * a];
    L.bc[2 * a + 1] = b1 < gn[a] - 1 ? BC_EXCHANGE : d->bc[2 * a + 1];
    L.lo[a] = (L.per[a] || L.bc[2 * a] == BC_EXCHANGE) ? 0 : 1;
    L.hi[a] = L.per[a] ? L.pn[a] - 1 : (L.bc[2 * a + 1] == BC_EXCHANGE ? L.n[a] - 1 : L.n[a] - 2);
  }
  L.cyl = d->geom == JZ_GEOM_CYLINDER;
  L.pitch = ((L.n[0] + 2 * NG) + 31) / 32 * 32;
  L.plane = (long long)L.pitch * (L.n[1] + 2 * NG);
  L.npad = L.plane * (L.n[2] + 2 * NG);
  c.es = d->precision == JZ_P64 ? 8 : 4;
  c.ms = (d->precision == JZ_P32 || d->precision == JZ_P32_S64) ? 4 : 8;
  c.tab_len = 0;
  for (int a = 0; a < 3; ++a) c.tab_len += 5 * (size_t)(L.n[a] + 2 * NG);
  c.tab_len += 2 * (size_t)(L.n[2] + 2 * NG);  // azimuth cos / sin
  size_t off = 0;
  c.off_sc = off; off = align256(off + sizeof(Scalars));
  // time-step rate partials, then the diagnostics records (RED_BLOCKS each)
  c.off_partial = off; off = align256(off + sizeof(double) * RED_BLOCKS * (DIAG_WORDS + 1));
  c.off_tab = off; off = align256(off + sizeof(double) * c.tab_len);
  c.off_inflow = off; off = align256(off + sizeof(double) * (size_t)L.n[1] * (size_t)L.n[2]);
  c.off_axis = off; off = align256(off + sizeof(double) * 5 * (size_t)(L.cyl ? L.n[0] : 1));
  size_t qbytes = align256(5 * (size_t)L.npad * c.es);
  c.off_q0 = off; off += qbytes;
  c.off_qa = off; off += qbytes;
  c.off_qb = off; off += qbytes;
  c.off_m = off; off += align256(10 * (size_t)L.npad * c.ms);
  c.off_q0d = off;  // FP64 state of a JZ_P32_S64 grid
  if (d->precision == JZ_P32_S64) off += align256(5 * (size_t)L.npad * 8);
  c.total = off;
  return c;
}

struct EventPair { cudaEvent_t a, b; int cls; };

int device_sm_count() {
  static std::atomic<int> cache[64];  // 0: not queried yet
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 1;
  if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

}  // namespace jz

using namespace jz;

struct jz_grid {
  jz_grid_desc desc;     // of the whole grid (a block: the grid it is part of)
  int o0[3], o1[3];      // the nodes of that grid held here (the whole grid: 0 .. n-1)
  jz_flow_params flow;
  bool have_flow = false;
  cudaStream_t stream = nullptr;
  Carve cv;
  GridDev dev;
  char* base = nullptr;
  // graph of one step
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  double graph_cfl = -1.0, graph_dt = -1.0;
  uint64_t graph_kernels = 0;
  // profiling
  bool profiling = false;
  std::vector<EventPair> events;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t handoff = nullptr;  // orders a new stream after the old one (jz_set_stream)
};

struct jz_batch {
  std::vector<jz_grid*> grids;
  bool coupled = false;         // blocks of one grid: halo exchange and one time step
  size_t off_x = 0;             // exchange entries, ordered by direction
  int xbegin[3] = {0, 0, 0}, xcount[3] = {0, 0, 0}, xblocks = 1;
  cudaStream_t stream = nullptr;
  int prec = 0;
  char* dev = nullptr;
  size_t off_stage = 0, off_bc = 0, off_rate = 0, off_items = 0, off_queue = 0, off_bcitems = 0;
  int nitems = 0, nbcitems = 0;
  int model = 0;                // stage kernel flow model shared by every grid (else the runtime model)
  bool cyl = false;             // some grid is cylindrical (centreline means before each boundary pass)
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  double graph_cfl = -1.0;
  uint64_t graph_kernels = 0;
};

namespace {

cudaEvent_t take_event(jz_grid* g) {
  if (!g->pool.empty()) {
    cudaEvent_t e = g->pool.back();
    g->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Enqueue `fn` (a launch) with optional profiling events around it.
template <typename Fn>
int timed(jz_grid* g, int cls, Fn fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (g->profiling) {
    a = take_event(g);
    b = take_event(g);
    if (!a || !b) return fail(JZ_ECUDA, "cudaEventCreate failed");
    JZ_CUDA(cudaEventRecord(a, g->stream));
  }
  cudaError_t e = fn();
  if (e != cudaSuccess) return fail(JZ_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
  if (g->profiling) {
    JZ_CUDA(cudaEventRecord(b, g->stream));
    g->events.push_back({a, b, cls});
  }
  return JZ_OK;
}

int enqueue_step(jz_grid* g, double cfl, double dt_fixed) {
  GridDev& d = g->dev;
  cudaStream_t s = g->stream;
  int rc;
  if ((rc = timed(g, 2, [&] { return launch_timestep(d, cfl, dt_fixed, s); }))) return rc;
  const int src[5] = {0, 1, 2, 1, 2};  // Q^(l-1): Q0, QA, QB, QA, QB
  const int out[5] = {1, 2, 1, 2, 0};  // Q^(l):   QA, QB, QA, QB, Q0
  void* dst[5] = {d.QA, d.QB, d.QA, d.QB, d.Q0};
  for (int l = 0; l < 5; ++l) {
    if ((rc = timed(g, 0, [&] { return launch_stage(d, l, src[l], out[l], s); }))) return rc;
    if ((rc = timed(g, 1, [&] { return launch_bc(d, dst[l], s); }))) return rc;
  }
  return JZ_OK;
}

int check_grid(jz_grid* g, bool need_flow) {
  if (!g) return fail(JZ_EINVAL, "null grid");
  if (need_flow && !g->have_flow) return fail(JZ_EINVAL, "flow parameters not set (call jz_state_init first)");
  return JZ_OK;
}

int check_dt(double cfl, double dt_fixed) {
  bool a = cfl > 0.0 && std::isfinite(cfl), b = dt_fixed > 0.0 && std::isfinite(dt_fixed);
  if (a == b) return fail(JZ_EINVAL, "exactly one of cfl (%g) and dt_fixed (%g) must be positive", cfl, dt_fixed);
  return JZ_OK;
}

// planes per CTA chunk: minimise (waves of resident CTAs) x (planes + prologue)
int default_kc(const Layout& L, StageTiling t, int ctas_per_sm) {
  long long tiles = (long long)((L.hi[0] + t.ti) / t.ti) * ((L.hi[1] + t.tj) / t.tj);
  int nz = L.hi[2] - L.lo[2] + 1;
  long long slots = (long long)device_sm_count() * ctas_per_sm;
  int best = nz;
  double best_cost = 1e300;
  for (int kc = 1; kc <= nz; ++kc) {
    long long ctas = tiles * ((nz + kc - 1) / kc);
    long long waves = (ctas + slots - 1) / slots;
    double cost = (double)waves * (kc + 3.0);
    if (cost < best_cost - 1e-9) { best_cost = cost; best = kc; }
  }
  return best;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 4-D map over a field array [fields][k][j][i-row of pitch]: box = one plane of
// (ti+4) x (tj+4) nodes (tile plus two-node halo) x all fields.  Coordinates
// outside the array read as zero.
int make_plane_map(CUtensorMap* m, void* base, bool fp64, const Layout& L, int fields, StageTiling t,
                   int halo_rows = 2) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(JZ_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  const size_t es = fp64 ? 8 : 4;
  // x extent: the row's nodes from ghost -2 to ghost n+1, not the padded
  // pitch, so that a tile box reaching past the grid's last ghost column
  // (ragged tiles of narrow grids) is zero-filled instead of fetching the
  // row padding from memory.  L2 promotion of 64 B: a box row (20 or 36
  // elements from a 64-byte boundary) then fetches the sectors it needs plus
  // at most one; 128 B and 256 B promotion moved 5% more DRAM bytes per
  // stage on the 256x192x192 grid and the 64-grid batch, at the same time
  cuuint64_t dims[4] = {(cuuint64_t)(L.n[0] + 2 * NG), (cuuint64_t)(L.n[1] + 2 * NG), (cuuint64_t)(L.n[2] + 2 * NG),
                        (cuuint64_t)fields};
  cuuint64_t strides[3] = {(cuuint64_t)L.pitch * es, (cuuint64_t)L.plane * es, (cuuint64_t)L.npad * es};
  cuuint32_t box[4] = {(cuuint32_t)(t.ti + 4), (cuuint32_t)(t.tj + 2 * halo_rows), 1, (cuuint32_t)fields};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(m, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_64B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(JZ_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return JZ_OK;
}

// TMA maps of the states and metrics for the tile of the kernel the grid runs
int build_maps(GridDev& d) {
  const StageTiling t = grid_tiling(d);
  const bool st64 = d.prec == JZ_P64, mt64 = d.prec == JZ_P64 || d.prec == JZ_P32_M64;
  int rc;
  if ((rc = make_plane_map(&d.tmQ[0], d.Q0, st64, d.L, 5, t)) || (rc = make_plane_map(&d.tmQ[1], d.QA, st64, d.L, 5, t)) ||
      (rc = make_plane_map(&d.tmQ[2], d.QB, st64, d.L, 5, t)) || (rc = make_plane_map(&d.tmM, d.M, mt64, d.L, 10, t)) ||
      (rc = make_plane_map(&d.tmMv, d.M, mt64, d.L, 10, t, 1)) ||
      (rc = make_plane_map(&d.tmQ0u, d.Q0, st64, d.L, 5, t, 0)))
    return rc;
  return JZ_OK;
}

void drop_graph(jz_grid* g) {
  if (g->exec) { cudaGraphExecDestroy(g->exec); g->exec = nullptr; }
  if (g->graph) { cudaGraphDestroy(g->graph); g->graph = nullptr; }
  g->graph_cfl = g->graph_dt = -1.0;
}

}  // namespace

namespace {
int create_grid(const jz_grid_desc* desc, const int* o0, const int* o1, void* dev_buf, size_t bytes, void* stream,
                jz_grid** out);
}  // namespace

extern "C" {

int jz_last_error(char* buf, size_t len) {
  if (buf && len > 0) {
    size_t n = g_error.size() < len - 1 ? g_error.size() : len - 1;
    memcpy(buf, g_error.data(), n);
    buf[n] = 0;
  }
  return (int)g_error.size();
}

int jz_grid_bytes(const jz_grid_desc* desc, size_t* bytes) {
  int rc = validate(desc);
  if (rc) return rc;
  if (!bytes) return fail(JZ_EINVAL, "null output");
  *bytes = carve(desc).total;
  return JZ_OK;
}

int jz_block_bytes(const jz_grid_desc* desc, const int o0[3], const int o1[3], size_t* bytes) {
  int rc = validate(desc);
  if (!rc) rc = validate_block(desc, o0, o1);
  if (rc) return rc;
  if (!bytes) return fail(JZ_EINVAL, "null output");
  *bytes = carve(desc, o0, o1).total;
  return JZ_OK;
}

int jz_grid_create(const jz_grid_desc* desc, void* dev_buf, size_t bytes, void* stream, jz_grid** out) {
  return create_grid(desc, nullptr, nullptr, dev_buf, bytes, stream, out);
}

int jz_block_create(const jz_grid_desc* desc, const int o0[3], const int o1[3], void* dev_buf, size_t bytes,
                    void* stream, jz_grid** out) {
  int rc = validate(desc);
  if (!rc) rc = validate_block(desc, o0, o1);
  if (rc) return rc;
  return create_grid(desc, o0, o1, dev_buf, bytes, stream, out);
}

}  // extern "C"

namespace {

int create_grid(const jz_grid_desc* desc, const int* o0, const int* o1, void* dev_buf, size_t bytes, void* stream,
                jz_grid** out) {
  int rc = validate(desc);
  if (rc) return rc;
  if (!out) return fail(JZ_EINVAL, "null output");
  *out = nullptr;
  Carve cv = carve(desc, o0, o1);
  if (!dev_buf) return fail(JZ_EINVAL, "null device buffer");
  if (((uintptr_t)dev_buf & 255) != 0) return fail(JZ_EINVAL, "device buffer must be 256-byte aligned");
  if (bytes < cv.total) return fail(JZ_ENOMEM, "device buffer holds %zu bytes, grid needs %zu", bytes, cv.total);
  static bool configured = false;
  if (!configured) {
    JZ_CUDA(stage_configure());
    configured = true;
  }
  jz_grid* g = new (std::nothrow) jz_grid();
  if (!g) return fail(JZ_ENOMEM, "host allocation failed");
  g->desc = *desc;
  for (int a = 0; a < 3; ++a) {
    g->o0[a] = o0 ? o0[a] : 0;
    g->o1[a] = o1 ? o1[a] : (a == 0 ? desc->ni : a == 1 ? desc->nj : desc->nk) - 1;
  }
  g->stream = (cudaStream_t)stream;
  g->cv = cv;
  g->base = (char*)dev_buf;
  GridDev& d = g->dev;
  d.L = cv.L;
  d.prec = desc->precision;
  d.Q0 = g->base + cv.off_q0;
  d.QA = g->base + cv.off_qa;
  d.QB = g->base + cv.off_qb;
  d.M = g->base + cv.off_m;
  d.Q0d = d.prec == JZ_P32_S64 ? (double*)(g->base + cv.off_q0d) : nullptr;
  d.sc = (Scalars*)(g->base + cv.off_sc);
  d.partial = (double*)(g->base + cv.off_partial);
  d.inflow = (double*)(g->base + cv.off_inflow);
  d.axis = (double*)(g->base + cv.off_axis);
  d.variant = d.prec == JZ_P32 ? 2 : 0;  // P32: the vector-record kernel (fastest measured)
  d.vti = 16;  // two CTAs per SM; as fast as 32 x 16 on 256x192x192, faster on small grids
  d.vtj = 16;
  d.kc = default_kc(cv.L, grid_tiling(d), grid_ctas_per_sm(d));
  const int gn[3] = {desc->ni, desc->nj, desc->nk};
  for (int a = 0; a < 3; ++a) {
    d.goff[a] = g->o0[a];
    d.gn[a] = gn[a];
  }
  memset(&d.F, 0, sizeof(d.F));
  // coordinate tables
  double* tab = (double*)(g->base + cv.off_tab);
  long long off = 0;
  for (int a = 0; a < 3; ++a) {
    d.C.base[a] = tab + off; off += cv.L.n[a] + 2 * NG;
    d.C.h[a] = tab + off; off += cv.L.n[a] + 2 * NG;
  }
  for (int a = 0; a < 3; ++a)
    for (int e = 0; e < 3; ++e) { d.C.sn[a][e] = tab + off; off += cv.L.n[e] + 2 * NG; }
  d.C.cth = tab + off; off += cv.L.n[2] + 2 * NG;
  d.C.sth = tab + off; off += cv.L.n[2] + 2 * NG;
  d.C.amp = desc->map_amp;
  d.C.cyl = cv.L.cyl;
  TabParams tp;
  for (int a = 0; a < 3; ++a) {
    tp.n[a] = cv.L.n[a];
    tp.off[a] = d.goff[a];
    tp.gn[a] = d.gn[a];
    tp.per[a] = cv.L.per[a];
    tp.pn[a] = cv.L.pn[a];
    tp.lo[a] = desc->lo[a];
    tp.hi[a] = desc->hi[a];
  }
  tp.cyl = cv.L.cyl;
  tp.cluster_r = desc->cluster_r;
  tp.stretch_c = desc->stretch_c;
  tp.stretch_w = desc->stretch_w;
  tp.amp = desc->map_amp;
  // mapping wave numbers (1..3) and phases drawn from SplitMix64(map_seed ^ c)
  for (int a = 0; a < 3; ++a)
    for (int e = 0; e < 3; ++e) {
      uint64_t c = (uint64_t)(3 * a + e);
      tp.m[3 * a + e] = 1 + (int)(splitmix64(desc->map_seed ^ (2 * c)) % 3ULL);
      tp.th[3 * a + e] = 2.0 * 3.14159265358979323846 * unit53(splitmix64(desc->map_seed ^ (2 * c + 1)));
    }
  if ((rc = build_maps(d))) {
    delete g;
    return rc;
  }
  cudaError_t e;
  if ((e = cudaMemsetAsync(d.sc, 0, sizeof(Scalars), g->stream)) != cudaSuccess ||
      (e = launch_tables(tp, tab, g->stream)) != cudaSuccess || (e = launch_metrics(d, g->stream)) != cudaSuccess) {
    delete g;
    return fail(JZ_ECUDA, "grid set-up failed: %s", cudaGetErrorString(e));
  }
  *out = g;
  return JZ_OK;
}

}  // namespace

extern "C" {

int jz_grid_destroy(jz_grid* g) {
  if (!g) return JZ_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (auto& p : g->events) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : g->pool) cudaEventDestroy(e);
  if (g->handoff) cudaEventDestroy(g->handoff);
  delete g;
  return JZ_OK;
}

int jz_set_stream(jz_grid* g, void* stream) {
  if (int rc = check_grid(g, false)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (s == g->stream) return JZ_OK;
  if (!g->handoff) JZ_CUDA(cudaEventCreateWithFlags(&g->handoff, cudaEventDisableTiming));
  JZ_CUDA(cudaEventRecord(g->handoff, g->stream));
  JZ_CUDA(cudaStreamWaitEvent(s, g->handoff, 0));
  g->stream = s;
  return JZ_OK;
}

// After a new state: the boundary pass over both ghost layers, then the
// whole padded arrays of Q^n copied into the two stage buffers, so that the
// second ghost layer behind physical faces, which the per-stage passes leave
// alone, holds finite values in every buffer (no updated node depends on it).
static int set_state_ghosts(jz_grid* g) {
  JZ_CUDA(launch_bc(g->dev, g->dev.Q0, g->stream, true));
  const size_t bytes = 5 * (size_t)g->dev.L.npad * (g->dev.prec == JZ_P64 ? 8 : 4);
  JZ_CUDA(cudaMemcpyAsync(g->dev.QA, g->dev.Q0, bytes, cudaMemcpyDeviceToDevice, g->stream));
  JZ_CUDA(cudaMemcpyAsync(g->dev.QB, g->dev.Q0, bytes, cudaMemcpyDeviceToDevice, g->stream));
  return JZ_OK;
}

int jz_state_init(jz_grid* g, const jz_flow_params* f, uint64_t seed) {
  if (int rc = check_grid(g, false)) return rc;
  if (!f) return fail(JZ_EINVAL, "null flow parameters");
  if (!(f->gamma > 1.0) || !(f->pr > 0.0) || !(f->prt > 0.0) || !(f->mach >= 0.0) || !(f->k2 >= 0.0) ||
      !(f->k4 >= 0.0) || !(f->sigma > 0.0) || !(f->s1 > 0.0) || !(f->cs >= 0.0) || !(f->theta > 0.0) ||
      !std::isfinite(f->re) || (f->ic != JZ_IC_JET && f->ic != JZ_IC_QUIESCENT) ||
      (f->sgs != JZ_SGS_SMAGORINSKY && f->sgs != JZ_SGS_VREMAN))
    return fail(JZ_EINVAL, "bad flow parameters");
  g->flow = *f;
  g->have_flow = true;
  FlowC& F = g->dev.F;
  F.gamma = f->gamma;
  F.gm1 = f->gamma - 1.0;
  F.cp = 1.0 / (f->gamma - 1.0);
  F.mu_inf = f->re > 0.0 ? f->mach / f->re : 0.0;
  F.s1 = f->s1;
  F.pr = f->pr;
  F.prt = f->prt;
  F.cs = f->cs;
  F.k2 = f->k2;
  F.k4 = f->k4;
  F.sigma = f->sigma;
  F.mach = f->mach;
  F.r0 = f->r0;
  F.theta = f->theta;
  F.noise = f->noise;
  F.ic = f->ic;
  F.sgs = f->sgs;
  F.viscous = (F.mu_inf > 0.0 || F.cs > 0.0) ? 1 : 0;
  F.vfac = std::fmax(4.0 / 3.0, f->gamma / f->pr);
  F.gamma_f = (float)F.gamma;
  F.gm1_f = (float)F.gm1;
  F.pe_f = (float)(1.0 / F.gamma);
  F.vfac_f = (float)F.vfac;
  if (g->exec) { cudaGraphExecDestroy(g->exec); g->exec = nullptr; }
  if (g->graph) { cudaGraphDestroy(g->graph); g->graph = nullptr; }
  g->graph_cfl = g->graph_dt = -1.0;
  JZ_CUDA(cudaMemsetAsync(g->dev.sc, 0, sizeof(Scalars), g->stream));
  JZ_CUDA(launch_init(g->dev, seed, g->stream));
  return set_state_ghosts(g);
}

int jz_rk_step(jz_grid* g, double cfl, double dt_fixed) {
  if (int rc = check_grid(g, true)) return rc;
  if (int rc = check_dt(cfl, dt_fixed)) return rc;
  return enqueue_step(g, cfl > 0.0 ? cfl : 0.0, dt_fixed);
}

int jz_nsteps(jz_grid* g, int n, double cfl, double dt_fixed) {
  if (int rc = check_grid(g, true)) return rc;
  if (int rc = check_dt(cfl, dt_fixed)) return rc;
  if (n < 0) return fail(JZ_EINVAL, "negative step count");
  if (n == 0) return JZ_OK;
  cfl = cfl > 0.0 ? cfl : 0.0;
  if (g->stream == nullptr || g->profiling) {  // the legacy stream cannot be captured
    for (int s = 0; s < n; ++s)
      if (int rc = enqueue_step(g, cfl, dt_fixed)) return rc;
    return JZ_OK;
  }
  if (!g->exec || g->graph_cfl != cfl || g->graph_dt != dt_fixed) {
    if (g->exec) { cudaGraphExecDestroy(g->exec); g->exec = nullptr; }
    if (g->graph) { cudaGraphDestroy(g->graph); g->graph = nullptr; }
    uint64_t before = g_launches.load();
    JZ_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step(g, cfl, dt_fixed);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
    g_launches.store(before);  // captured launches are counted when replayed
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return fail(JZ_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    g->graph = graph;
    JZ_CUDA(cudaGraphInstantiate(&g->exec, graph, 0));
    size_t nodes = 0;
    JZ_CUDA(cudaGraphGetNodes(graph, nullptr, &nodes));
    g->graph_kernels = nodes;
    g->graph_cfl = cfl;
    g->graph_dt = dt_fixed;
  }
  for (int s = 0; s < n; ++s) JZ_CUDA(cudaGraphLaunch(g->exec, g->stream));
  count_launches((uint64_t)n * g->graph_kernels);
  return JZ_OK;
}

int jz_diagnostics(jz_grid* g, jz_diag* out) {
  if (int rc = check_grid(g, true)) return rc;
  if (!out) return fail(JZ_EINVAL, "null output");
  JZ_CUDA(launch_diagnostics(g->dev, g->stream));
  Scalars h;
  JZ_CUDA(cudaMemcpyAsync(&h, g->dev.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, g->stream));
  JZ_CUDA(cudaStreamSynchronize(g->stream));
  out->time = h.time;
  out->step = h.step;
  out->dt = h.dt;
  for (int v = 0; v < 5; ++v) out->sum[v] = h.diag[v];
  out->rho_min = h.diag[5];
  out->rho_max = h.diag[6];
  out->p_min = h.diag[7];
  out->p_max = h.diag[8];
  out->mach_max = h.diag[9];
  out->nonfinite = (int64_t)h.diag[10];
  if (h.err)
    return fail(JZ_ETIMEOUT,
                "a bounded device wait gave up (stage kernel data staging: barrier %d parity %d plane %d tile %d,%d "
                "chunk %d input %d); results are invalid",
                h.errinfo[0], h.errinfo[1], h.errinfo[2], h.errinfo[3], h.errinfo[4], h.errinfo[5], h.errinfo[6]);
  if (out->nonfinite > 0) return fail(JZ_ENONFINITE, "%lld grid nodes hold non-finite values", (long long)out->nonfinite);
  return JZ_OK;
}

int jz_diagnostics_async(jz_grid* g, jz_diag* out) {
  if (int rc = check_grid(g, true)) return rc;
  if (!out) return fail(JZ_EINVAL, "null output");
  JZ_CUDA(launch_diagnostics(g->dev, g->stream));
  JZ_CUDA(cudaMemcpyAsync(out, &g->dev.sc->out, sizeof(jz_diag), cudaMemcpyDeviceToHost, g->stream));
  return JZ_OK;
}

int jz_set_step_diagnostics(jz_grid* g, int on) {
  if (int rc = check_grid(g, false)) return rc;
  if (on != 0 && on != 1) return fail(JZ_EINVAL, "step diagnostics flag must be 0 or 1");
  if (g->dev.step_diag != on) {
    g->dev.step_diag = on;
    drop_graph(g);  // captured launches carry the flag
  }
  return JZ_OK;
}

int jz_step_diagnostics_async(jz_grid* g, jz_diag* out) {
  if (int rc = check_grid(g, false)) return rc;
  if (!out) return fail(JZ_EINVAL, "null output");
  JZ_CUDA(cudaMemcpyAsync(out, &g->dev.sc->out, sizeof(jz_diag), cudaMemcpyDeviceToHost, g->stream));
  return JZ_OK;
}

static size_t state_count(const jz_grid* g) {
  const Layout& L = g->dev.L;  // the grid's (a block's) own nodes
  return 5ULL * (size_t)L.n[0] * (size_t)L.n[1] * (size_t)L.n[2];
}

int jz_state_download(jz_grid* g, double* host, size_t n) {
  if (int rc = check_grid(g, false)) return rc;
  if (!host) return fail(JZ_EINVAL, "null host buffer");
  if (n != state_count(g)) return fail(JZ_EINVAL, "host buffer holds %zu values, state has %zu", n, state_count(g));
  double* staging = (double*)g->dev.QA;  // QA and QB are free between steps
  JZ_CUDA(launch_pack(g->dev, staging, g->stream));
  JZ_CUDA(cudaMemcpyAsync(host, staging, n * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  JZ_CUDA(cudaStreamSynchronize(g->stream));
  return JZ_OK;
}

int jz_metrics_download(jz_grid* g, double* host, size_t n) {
  if (int rc = check_grid(g, false)) return rc;
  if (!host) return fail(JZ_EINVAL, "null host buffer");
  const size_t N = state_count(g) / 5;
  if (n != 10 * N) return fail(JZ_EINVAL, "host buffer holds %zu values, metrics have %zu", n, 10 * N);
  double* staging = (double*)g->dev.QA;  // one FP64 field fits the free stage buffer QA
  for (int f = 0; f < 10; ++f) {
    JZ_CUDA(launch_pack_metric(g->dev, f, staging, g->stream));
    JZ_CUDA(cudaMemcpyAsync(host + (size_t)f * N, staging, N * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  }
  JZ_CUDA(cudaStreamSynchronize(g->stream));
  return JZ_OK;
}

int jz_state_upload(jz_grid* g, const double* host, size_t n) {
  if (int rc = check_grid(g, true)) return rc;
  if (!host) return fail(JZ_EINVAL, "null host buffer");
  if (n != state_count(g)) return fail(JZ_EINVAL, "host buffer holds %zu values, state has %zu", n, state_count(g));
  double* staging = (double*)g->dev.QA;
  JZ_CUDA(cudaMemcpyAsync(staging, host, n * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  JZ_CUDA(launch_unpack(g->dev, staging, g->stream));
  if (int rc = set_state_ghosts(g)) return rc;
  JZ_CUDA(cudaStreamSynchronize(g->stream));
  return JZ_OK;
}

int jz_launch_count(uint64_t* out) {
  if (!out) return fail(JZ_EINVAL, "null output");
  *out = g_launches.load();
  return JZ_OK;
}

int jz_profile_begin(jz_grid* g) {
  if (int rc = check_grid(g, false)) return rc;
  for (auto& p : g->events) { g->pool.push_back(p.a); g->pool.push_back(p.b); }
  g->events.clear();
  g->profiling = true;
  return JZ_OK;
}

int jz_profile_read(jz_grid* g, double ms[4], int64_t launches[4]) {
  if (int rc = check_grid(g, false)) return rc;
  if (!ms || !launches) return fail(JZ_EINVAL, "null output");
  JZ_CUDA(cudaStreamSynchronize(g->stream));
  for (int c = 0; c < 4; ++c) { ms[c] = 0.0; launches[c] = 0; }
  for (auto& p : g->events) {
    float t = 0.f;
    JZ_CUDA(cudaEventElapsedTime(&t, p.a, p.b));
    ms[p.cls] += t;
    launches[p.cls] += 1;
  }
  return JZ_OK;
}

int jz_profile_end(jz_grid* g) {
  if (int rc = check_grid(g, false)) return rc;
  g->profiling = false;
  for (auto& p : g->events) { g->pool.push_back(p.a); g->pool.push_back(p.b); }
  g->events.clear();
  return JZ_OK;
}

int jz_get_tiling(jz_grid* g, int* ti, int* tj, int* kc) {
  if (int rc = check_grid(g, false)) return rc;
  StageTiling t = grid_tiling(g->dev);
  if (ti) *ti = t.ti;
  if (tj) *tj = t.tj;
  if (kc) *kc = g->dev.kc;
  return JZ_OK;
}

int jz_set_stage_variant(jz_grid* g, int variant) {
  if (int rc = check_grid(g, false)) return rc;
  if (variant != 0 && variant != 2) return fail(JZ_EINVAL, "stage variant must be 0 or 2");
  if (variant != 0 && g->dev.prec != JZ_P32) return fail(JZ_EINVAL, "stage variant 2 is FP32 (JZ_P32) only");
  g->dev.variant = variant;
  drop_graph(g);
  return build_maps(g->dev);  // the two kernels may stage different tiles
}

// --- a block of a grid partitioned over ranks ------------------------------

static int halo_args(jz_grid* g, int which, int dir, int side) {
  if (int rc = check_grid(g, false)) return rc;
  if (which < 0 || which > 2) return fail(JZ_EINVAL, "state copy %d is not 0 (Q0), 1 (QA) or 2 (QB)", which);
  if (dir < 0 || dir > 2 || side < 0 || side > 1) return fail(JZ_EINVAL, "bad face (direction %d, side %d)", dir, side);
  if (g->dev.L.bc[2 * dir + side] != BC_EXCHANGE)
    return fail(JZ_EINVAL, "face (direction %d, side %d) is not an exchange face of this block", dir, side);
  return JZ_OK;
}

static void* state_copy(GridDev& d, int which) { return which == 0 ? d.Q0 : (which == 1 ? d.QA : d.QB); }

int jz_halo_bytes(jz_grid* g, int dir, size_t* bytes) {
  if (int rc = check_grid(g, false)) return rc;
  if (dir < 0 || dir > 2 || !bytes) return fail(JZ_EINVAL, "bad direction %d or null output", dir);
  const Layout& L = g->dev.L;
  const int e1 = dir == 0 ? 1 : 0, e2 = dir == 2 ? 1 : 2;
  *bytes = 10ULL * (size_t)(L.n[e1] + 2 * NG) * (size_t)(L.n[e2] + 2 * NG) * (g->dev.prec == JZ_P64 ? 8 : 4);
  return JZ_OK;
}

int jz_halo_pack(jz_grid* g, int which, int dir, int side, void* buf) {
  if (int rc = halo_args(g, which, dir, side)) return rc;
  if (!buf) return fail(JZ_EINVAL, "null halo buffer");
  const int first = side == 0 ? 0 : g->dev.L.n[dir] - 2;
  JZ_CUDA(launch_halo(g->dev, state_copy(g->dev, which), buf, dir, first, true, g->stream));
  return JZ_OK;
}

int jz_halo_unpack(jz_grid* g, int which, int dir, int side, const void* buf) {
  if (int rc = halo_args(g, which, dir, side)) return rc;
  if (!buf) return fail(JZ_EINVAL, "null halo buffer");
  const int first = side == 0 ? -NG : g->dev.L.n[dir];
  JZ_CUDA(launch_halo(g->dev, state_copy(g->dev, which), const_cast<void*>(buf), dir, first, false, g->stream));
  return JZ_OK;
}

int jz_block_rate(jz_grid* g, double** dev_rate) {
  if (int rc = check_grid(g, true)) return rc;
  if (!dev_rate) return fail(JZ_EINVAL, "null output");
  JZ_CUDA(launch_rate(g->dev, g->stream));
  *dev_rate = &g->dev.sc->rate;
  return JZ_OK;
}

int jz_block_advance(jz_grid* g, double cfl) {
  if (int rc = check_grid(g, true)) return rc;
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return fail(JZ_EINVAL, "cfl must be positive and finite (%g)", cfl);
  JZ_CUDA(launch_advance_from_rate(g->dev, cfl, g->stream));
  return JZ_OK;
}

int jz_block_stage(jz_grid* g, int stage) {
  if (int rc = check_grid(g, true)) return rc;
  if (stage < 0 || stage > 4) return fail(JZ_EINVAL, "stage %d is not 0..4", stage);
  GridDev& d = g->dev;
  const int src[5] = {0, 1, 2, 1, 2}, out[5] = {1, 2, 1, 2, 0};
  JZ_CUDA(launch_stage(d, stage, src[stage], out[stage], g->stream));
  JZ_CUDA(launch_bc(d, state_copy(d, out[stage]), g->stream));
  return JZ_OK;
}

int jz_set_stall_test(jz_grid* g, int on) {
  if (int rc = check_grid(g, false)) return rc;
  if (on != 0 && on != 1) return fail(JZ_EINVAL, "stall test flag must be 0 or 1");
  g->dev.stall_test = on;
  drop_graph(g);  // captured launches carry the flag
  return JZ_OK;
}

int jz_set_tile_shape(jz_grid* g, int ti, int tj) {
  if (int rc = check_grid(g, false)) return rc;
  if (g->dev.prec != JZ_P32 || g->dev.variant != 2)
    return fail(JZ_EINVAL, "the tile shape is chosen for the FP32 vector-record kernel only (JZ_P32, variant 2)");
  if (!((ti == 32 && tj == 16) || (ti == 16 && tj == 32) || (ti == 16 && tj == 16)))
    return fail(JZ_EINVAL, "tile shape %d x %d is not one of 32 x 16, 16 x 32, 16 x 16", ti, tj);
  g->dev.vti = ti;
  g->dev.vtj = tj;
  g->dev.kc = default_kc(g->dev.L, grid_tiling(g->dev), grid_ctas_per_sm(g->dev));
  drop_graph(g);
  return build_maps(g->dev);
}

int jz_set_tiling(jz_grid* g, int kc) {
  if (int rc = check_grid(g, false)) return rc;
  if (kc < 1) return fail(JZ_EINVAL, "kc must be >= 1");
  g->dev.kc = kc;
  drop_graph(g);
  return JZ_OK;
}

// ---- batches: many grids per launch ----------------------------------------

}  // extern "C"

namespace {

struct BatchPlan {
  size_t off_stage, off_bc, off_rate, off_items, off_queue, off_x, off_bcitems, total;
  std::vector<int4> items;
  std::vector<int4> bcitems;  // boundary-pass work items
  std::vector<XEntry> xs;  // halo exchange (blocks of one grid)
  int xbegin[3] = {0, 0, 0}, xcount[3] = {0, 0, 0}, xblocks = 1;
};

// Work items (grid, tile x, tile y, k-chunk) of every grid, and the layout
// of the batch's device tables.  Grids are queued largest first (total
// work), and the items of one grid stay together in row-major tile order:
// CTAs then take neighbouring tiles of a grid at the same time, so the halo
// rows two tiles share are read from memory once and served from L2 to the
// second (sorting single items by size scattered a grid's ragged edge tiles
// to the end of the queue and read their halos twice).
int batch_plan(jz_grid* const* grids, int n, BatchPlan& P) {
  if (!grids || n < 1) return fail(JZ_EINVAL, "bad batch arguments");
  int prec = -1;
  for (int k = 0; k < n; ++k) {
    if (int rc = check_grid(grids[k], true)) return rc;
    if (prec >= 0 && grids[k]->dev.prec != prec) return fail(JZ_EINVAL, "batch grids must share one precision mode");
    prec = grids[k]->dev.prec;
  }
  const StageTiling t = grid_tiling(grids[0]->dev);
  for (int k = 1; k < n; ++k) {
    const StageTiling u = grid_tiling(grids[k]->dev);
    if (grids[k]->dev.variant != grids[0]->dev.variant || u.ti != t.ti || u.tj != t.tj)
      return fail(JZ_EINVAL, "batch grids must share one stage kernel and tile shape");
  }
  std::vector<std::pair<long long, std::vector<int4>>> work;  // (grid's total cost, its items)
  for (int k = 0; k < n; ++k) {
    work.push_back({0, {}});
    const Layout& L = grids[k]->dev.L;
    const int kc = grids[k]->dev.kc;
    const int tx = (L.hi[0] + t.ti) / t.ti, ty = (L.hi[1] + t.tj) / t.tj;
    const int nz = L.hi[2] - L.lo[2] + 1, cz = (nz + kc - 1) / kc;
    for (int bz = 0; bz < cz; ++bz) {
      const int planes = (bz + 1) * kc <= nz ? kc : nz - bz * kc;
      for (int by = 0; by < ty; ++by)
        for (int bx = 0; bx < tx; ++bx) {
          const int ox = std::min(L.hi[0], (bx + 1) * t.ti - 1) - std::max(L.lo[0], bx * t.ti) + 1;
          const int oy = std::min(L.hi[1], (by + 1) * t.tj - 1) - std::max(L.lo[1], by * t.tj) + 1;
          work.back().first += (long long)(planes + 3) * (ox > 0 ? ox : 0) * (oy > 0 ? oy : 0) + 1;
          work.back().second.push_back(make_int4(k, bx, by, bz));
        }
    }
  }
  std::stable_sort(work.begin(), work.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  P.items.clear();
  for (auto& w : work) P.items.insert(P.items.end(), w.second.begin(), w.second.end());
  size_t off = 0;
  P.off_stage = off; off = align256(off + (size_t)n * stage_ctx_bytes(prec));
  P.off_bc = off; off = align256(off + (size_t)n * bc_ctx_bytes());
  P.off_rate = off; off = align256(off + (size_t)n * rate_ctx_bytes());
  P.off_items = off; off = align256(off + P.items.size() * sizeof(int4));
  P.off_queue = off; off = align256(off + sizeof(unsigned int));
  P.off_x = off; off = align256(off + P.xs.size() * sizeof(XEntry));
  P.bcitems.clear();
  for (int k = 0; k < n; ++k) bc_fill_items(grids[k]->dev, k, P.bcitems);
  P.off_bcitems = off; off = align256(off + P.bcitems.size() * sizeof(int4));
  P.total = off;
  return JZ_OK;
}

// Blocks of one grid: same grid description, a partition of its nodes, and
// for every exchange face exactly one neighbour sharing the face over the
// same node ranges.  Fills the exchange entries (direction order) and then
// the batch plan.
int blocks_plan(jz_grid* const* grids, int n, BatchPlan& P) {
  if (!grids || n < 1) return fail(JZ_EINVAL, "bad block-set arguments");
  for (int k = 0; k < n; ++k)
    if (int rc = check_grid(grids[k], true)) return rc;
  const jz_grid_desc& G = grids[0]->desc;
  const int gn[3] = {G.ni, G.nj, G.nk};
  long long nodes = 0;
  for (int k = 0; k < n; ++k) {
    if (memcmp(&grids[k]->desc, &G, sizeof(G)) != 0) return fail(JZ_EINVAL, "blocks %d and 0 describe different grids", k);
    long long v = 1;
    for (int a = 0; a < 3; ++a) v *= grids[k]->o1[a] - grids[k]->o0[a] + 1;
    nodes += v;
  }
  if (nodes != (long long)gn[0] * gn[1] * gn[2]) return fail(JZ_EINVAL, "the blocks do not partition the grid's nodes");
  std::vector<XEntry> byd[3];
  long long biggest = 1;
  for (int k = 0; k < n; ++k) {
    const jz_grid* A = grids[k];
    for (int d = 0; d < 3; ++d)
      for (int side = 0; side < 2; ++side) {
        if (A->dev.L.bc[2 * d + side] != BC_EXCHANGE) continue;
        // the neighbour starts right after A (side 1) or ends right before it (side 0)
        int found = -1;
        for (int m = 0; m < n && found < 0; ++m) {
          const jz_grid* B = grids[m];
          bool ok = side ? B->o0[d] == A->o1[d] + 1 : B->o1[d] == A->o0[d] - 1;
          for (int e = 0; e < 3 && ok; ++e)
            if (e != d) ok = B->o0[e] == A->o0[e] && B->o1[e] == A->o1[e];
          if (ok) found = m;
        }
        if (found < 0)
          return fail(JZ_EINVAL, "block %d: no neighbour shares its face %d%c over the same node ranges", k, d,
                      side ? '+' : '-');
        const jz_grid* B = grids[found];
        XEntry x;
        memset(&x, 0, sizeof(x));
        x.dq[0] = A->dev.Q0; x.dq[1] = A->dev.QA; x.dq[2] = A->dev.QB;
        x.sq[0] = B->dev.Q0; x.sq[1] = B->dev.QA; x.sq[2] = B->dev.QB;
        x.dpitch = A->dev.L.pitch; x.dplane = A->dev.L.plane; x.dnpad = A->dev.L.npad;
        x.spitch = B->dev.L.pitch; x.splane = B->dev.L.plane; x.snpad = B->dev.L.npad;
        x.d = d;
        x.dfirst = side ? A->dev.L.n[d] : -NG;
        x.sfirst = side ? 0 : B->dev.L.n[d] - NG;
        const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
        x.ea = A->dev.L.n[e1] + 2 * NG;
        x.eb = A->dev.L.n[e2] + 2 * NG;
        biggest = std::max(biggest, 10LL * x.ea * x.eb);
        byd[d].push_back(x);
      }
  }
  P.xs.clear();
  for (int d = 0; d < 3; ++d) {
    P.xbegin[d] = (int)P.xs.size();
    P.xcount[d] = (int)byd[d].size();
    P.xs.insert(P.xs.end(), byd[d].begin(), byd[d].end());
  }
  P.xblocks = (int)std::min<long long>((biggest + 255) / 256, 1024);
  return batch_plan(grids, n, P);
}

// halo exchange of state copy `which` between the blocks of a block set
int enqueue_exchange(jz_batch* b, int which) {
  for (int d = 0; d < 3; ++d) {
    cudaError_t e = launch_exchange(b->prec, b->dev + b->off_x, b->xbegin[d], b->xcount[d], b->xblocks, which, b->stream);
    if (e != cudaSuccess) return fail(JZ_ECUDA, "halo exchange launch failed: %s", cudaGetErrorString(e));
  }
  return JZ_OK;
}

int enqueue_batch_step(jz_batch* b, double cfl) {
  const int n = (int)b->grids.size();
  cudaStream_t s = b->stream;
  // blocks of one grid: Q^n's ghosts behind exchange faces first (its
  // boundary nodes and boundary ghosts are set by the previous fill)
  if (b->coupled)
    if (int rc = enqueue_exchange(b, 0)) return rc;
  cudaError_t e = launch_timestep_batch(b->prec, b->dev + b->off_rate, n, cfl, b->coupled, s);
  if (e != cudaSuccess) return fail(JZ_ECUDA, "batched time step launch failed: %s", cudaGetErrorString(e));
  const int src[5] = {0, 1, 2, 1, 2}, out[5] = {1, 2, 1, 2, 0};
  for (int l = 0; l < 5; ++l) {
    e = launch_stage_batch(b->prec, b->grids[0]->dev.variant, grid_tiling(b->grids[0]->dev), b->dev + b->off_stage,
                           (const int4*)(b->dev + b->off_items), b->nitems, (unsigned int*)(b->dev + b->off_queue), l,
                           src[l], out[l], b->model, s);
    if (e != cudaSuccess) return fail(JZ_ECUDA, "batched stage launch failed: %s", cudaGetErrorString(e));
    e = launch_bc_batch(b->prec, b->dev + b->off_bc, n, (const int4*)(b->dev + b->off_bcitems), b->nbcitems, out[l],
                        b->cyl, s);
    if (e != cudaSuccess) return fail(JZ_ECUDA, "batched boundary launch failed: %s", cudaGetErrorString(e));
    if (b->coupled && l < 4)
      if (int rc = enqueue_exchange(b, out[l])) return rc;
  }
  return JZ_OK;
}

// A batch (independent grids) or a block set (coupled: blocks of one grid).
int create_batch(jz_grid* const* grids, int n, bool coupled, void* dev_buf, size_t bytes, void* stream,
                 jz_batch** out) {
  if (!out) return fail(JZ_EINVAL, "null output");
  *out = nullptr;
  BatchPlan P;
  if (int rc = coupled ? blocks_plan(grids, n, P) : batch_plan(grids, n, P)) return rc;
  if (!dev_buf || ((uintptr_t)dev_buf & 255)) return fail(JZ_EINVAL, "batch buffer must be non-null and 256-byte aligned");
  if (bytes < P.total) return fail(JZ_ENOMEM, "batch buffer holds %zu bytes, batch needs %zu", bytes, P.total);
  const int prec = grids[0]->dev.prec;
  std::vector<char> host(P.total, 0);
  for (int k = 0; k < n; ++k) {
    stage_ctx_fill(host.data() + P.off_stage + (size_t)k * stage_ctx_bytes(prec), grids[k]->dev);
    bc_ctx_fill(host.data() + P.off_bc + (size_t)k * bc_ctx_bytes(), grids[k]->dev);
    rate_ctx_fill(host.data() + P.off_rate + (size_t)k * rate_ctx_bytes(), grids[k]->dev);
  }
  memcpy(host.data() + P.off_items, P.items.data(), P.items.size() * sizeof(int4));
  if (!P.xs.empty()) memcpy(host.data() + P.off_x, P.xs.data(), P.xs.size() * sizeof(XEntry));
  memcpy(host.data() + P.off_bcitems, P.bcitems.data(), P.bcitems.size() * sizeof(int4));
  JZ_CUDA(cudaMemcpy(dev_buf, host.data(), P.total, cudaMemcpyHostToDevice));
  jz_batch* b = new (std::nothrow) jz_batch();
  if (!b) return fail(JZ_ENOMEM, "host allocation failed");
  b->grids.assign(grids, grids + n);
  b->stream = (cudaStream_t)stream;
  b->prec = prec;
  b->dev = (char*)dev_buf;
  b->off_stage = P.off_stage;
  b->off_bc = P.off_bc;
  b->off_rate = P.off_rate;
  b->off_items = P.off_items;
  b->off_queue = P.off_queue;
  b->nitems = (int)P.items.size();
  b->off_bcitems = P.off_bcitems;
  b->nbcitems = (int)P.bcitems.size();
  for (int k = 0; k < n; ++k) b->cyl = b->cyl || grids[k]->dev.L.cyl;
  b->model = stage_model(grids[0]->dev);
  for (int k = 1; k < n; ++k)
    if (stage_model(grids[k]->dev) != b->model) b->model = 0;  // the runtime model serves a mix
  b->coupled = coupled;
  b->off_x = P.off_x;
  for (int d = 0; d < 3; ++d) {
    b->xbegin[d] = P.xbegin[d];
    b->xcount[d] = P.xcount[d];
  }
  b->xblocks = P.xblocks;
  *out = b;
  return JZ_OK;
}

}  // namespace

extern "C" {

int jz_batch_bytes(jz_grid* const* grids, int n, size_t* bytes) {
  if (!bytes) return fail(JZ_EINVAL, "null output");
  BatchPlan P;
  if (int rc = batch_plan(grids, n, P)) return rc;
  *bytes = P.total;
  return JZ_OK;
}

int jz_batch_create(jz_grid* const* grids, int n, void* dev_buf, size_t bytes, void* stream, jz_batch** out) {
  return create_batch(grids, n, false, dev_buf, bytes, stream, out);
}

int jz_blocks_bytes(jz_grid* const* blocks, int n, size_t* bytes) {
  if (!bytes) return fail(JZ_EINVAL, "null output");
  BatchPlan P;
  if (int rc = blocks_plan(blocks, n, P)) return rc;
  *bytes = P.total;
  return JZ_OK;
}

int jz_blocks_create(jz_grid* const* blocks, int n, void* dev_buf, size_t bytes, void* stream, jz_batch** out) {
  return create_batch(blocks, n, true, dev_buf, bytes, stream, out);
}

int jz_batch_nsteps(jz_batch* b, int n, double cfl) {
  if (!b) return fail(JZ_EINVAL, "null batch");
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return fail(JZ_EINVAL, "batch steps need a positive CFL number");
  if (n < 0) return fail(JZ_EINVAL, "negative step count");
  if (n == 0) return JZ_OK;
  if (b->stream == nullptr) {  // the legacy stream cannot be captured
    for (int s = 0; s < n; ++s)
      if (int rc = enqueue_batch_step(b, cfl)) return rc;
    return JZ_OK;
  }
  if (!b->exec || b->graph_cfl != cfl) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    uint64_t before = g_launches.load();
    JZ_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_batch_step(b, cfl);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    g_launches.store(before);
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return fail(JZ_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    b->graph = graph;
    JZ_CUDA(cudaGraphInstantiate(&b->exec, graph, 0));
    size_t nodes = 0;
    JZ_CUDA(cudaGraphGetNodes(graph, nullptr, &nodes));
    std::vector<cudaGraphNode_t> list(nodes);
    JZ_CUDA(cudaGraphGetNodes(graph, list.data(), &nodes));
    uint64_t kernels = 0;
    for (auto nd : list) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
    }
    b->graph_kernels = kernels;
    b->graph_cfl = cfl;
  }
  for (int s = 0; s < n; ++s) JZ_CUDA(cudaGraphLaunch(b->exec, b->stream));
  count_launches((uint64_t)n * b->graph_kernels);
  return JZ_OK;
}

int jz_batch_destroy(jz_batch* b) {
  if (!b) return JZ_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
  return JZ_OK;
}

// ---- time statistics -------------------------------------------------------

int jz_set_clock(jz_grid* g, double time, int64_t step) {
  if (int rc = check_grid(g, false)) return rc;
  if (!std::isfinite(time) || step < 0) return fail(JZ_EINVAL, "bad clock (time %g, step %lld)", time, (long long)step);
  Scalars* sc = g->dev.sc;
  JZ_CUDA(cudaMemcpyAsync(&sc->time, &time, sizeof(double), cudaMemcpyHostToDevice, g->stream));
  long long st = step;
  JZ_CUDA(cudaMemcpyAsync(&sc->step, &st, sizeof(long long), cudaMemcpyHostToDevice, g->stream));
  JZ_CUDA(cudaStreamSynchronize(g->stream));  // the host values go out of scope
  return JZ_OK;
}

}  // extern "C"

struct jz_stats {
  jz_grid* g = nullptr;
  double* su = nullptr;   // sum of u over samples, per node [k][j][i]
  double* su2 = nullptr;  // sum of u^2
  double* scr = nullptr;  // plane coordinates / axial coordinates
  int64_t samples = 0;
};

namespace {

struct StatsCarve { size_t off_su, off_su2, off_scr, total; };

StatsCarve stats_carve(const jz_grid* g) {
  const Layout& L = g->dev.L;
  const size_t N = (size_t)L.n[0] * L.n[1] * L.n[2];
  const size_t scr = std::max((size_t)2 * L.n[1] * L.n[2], (size_t)L.n[0]);
  StatsCarve c;
  size_t off = 0;
  c.off_su = off; off = align256(off + 8 * N);
  c.off_su2 = off; off = align256(off + 8 * N);
  c.off_scr = off; off = align256(off + 8 * scr);
  c.total = off;
  return c;
}

// plane index of the grid nodes nearest the axis along j or k: both
// middle nodes of an even count, the middle node of an odd one
void axis_nodes(int n, int c[2], int& m) {
  if (n % 2 == 0) { c[0] = n / 2 - 1; c[1] = n / 2; m = 2; }
  else { c[0] = c[1] = n / 2; m = 1; }
}

}  // namespace

extern "C" {

int jz_stats_bytes(jz_grid* g, size_t* bytes) {
  if (int rc = check_grid(g, false)) return rc;
  if (!bytes) return fail(JZ_EINVAL, "null output");
  *bytes = stats_carve(g).total;
  return JZ_OK;
}

int jz_stats_create(jz_grid* g, void* dev_buf, size_t bytes, jz_stats** out) {
  if (int rc = check_grid(g, false)) return rc;
  if (!out) return fail(JZ_EINVAL, "null output");
  *out = nullptr;
  const StatsCarve c = stats_carve(g);
  if (!dev_buf || ((uintptr_t)dev_buf & 255)) return fail(JZ_EINVAL, "statistics buffer must be non-null and 256-byte aligned");
  if (bytes < c.total) return fail(JZ_ENOMEM, "statistics buffer holds %zu bytes, needs %zu", bytes, c.total);
  jz_stats* s = new (std::nothrow) jz_stats();
  if (!s) return fail(JZ_ENOMEM, "host allocation failed");
  s->g = g;
  s->su = (double*)((char*)dev_buf + c.off_su);
  s->su2 = (double*)((char*)dev_buf + c.off_su2);
  s->scr = (double*)((char*)dev_buf + c.off_scr);
  if (cudaMemsetAsync(dev_buf, 0, c.off_scr, g->stream) != cudaSuccess) {
    delete s;
    return fail(JZ_ECUDA, "clearing the statistics failed");
  }
  *out = s;
  return JZ_OK;
}

int jz_stats_sample(jz_stats* s) {
  if (!s) return fail(JZ_EINVAL, "null statistics");
  JZ_CUDA(launch_stats_sample(s->g->dev, s->su, s->su2, s->g->stream));
  ++s->samples;
  return JZ_OK;
}

int jz_stats_count(jz_stats* s, int64_t* samples) {
  if (!s || !samples) return fail(JZ_EINVAL, "null argument");
  *samples = s->samples;
  return JZ_OK;
}

int jz_stats_read(jz_stats* s, double* mean_u, double* rms_u, size_t n) {
  if (!s || !mean_u || !rms_u) return fail(JZ_EINVAL, "null argument");
  const Layout& L = s->g->dev.L;
  const size_t N = (size_t)L.n[0] * L.n[1] * L.n[2];
  if (n != N) return fail(JZ_EINVAL, "host arrays hold %zu values, the grid has %zu nodes", n, N);
  if (s->samples < 1) return fail(JZ_EINVAL, "no samples");
  JZ_CUDA(cudaMemcpyAsync(mean_u, s->su, 8 * N, cudaMemcpyDeviceToHost, s->g->stream));
  JZ_CUDA(cudaMemcpyAsync(rms_u, s->su2, 8 * N, cudaMemcpyDeviceToHost, s->g->stream));
  JZ_CUDA(cudaStreamSynchronize(s->g->stream));
  const double ns = (double)s->samples;
  for (size_t t = 0; t < N; ++t) {
    const double m = mean_u[t] / ns;
    mean_u[t] = m;
    rms_u[t] = std::sqrt(std::max(rms_u[t] / ns - m * m, 0.0));
  }
  return JZ_OK;
}

int jz_stats_radial(jz_stats* s, double x, int nbins, double r_max, double* mean_u, double* rms_u, double* count) {
  if (!s || !mean_u || !rms_u || !count) return fail(JZ_EINVAL, "null argument");
  if (nbins < 1 || !(r_max > 0.0)) return fail(JZ_EINVAL, "need nbins >= 1 and r_max > 0");
  if (s->samples < 1) return fail(JZ_EINVAL, "no samples");
  const Layout& L = s->g->dev.L;
  const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
  cudaStream_t st = s->g->stream;
  // the plane whose axial coordinate (at the node nearest the axis) is nearest x
  int cj[2], ck[2], mj, mk;
  axis_nodes(n1, cj, mj);
  axis_nodes(n2, ck, mk);
  std::vector<double> xs(n0);
  JZ_CUDA(launch_stats_axis_x(s->g->dev, cj[0], ck[0], s->scr, st));
  JZ_CUDA(cudaMemcpyAsync(xs.data(), s->scr, 8 * (size_t)n0, cudaMemcpyDeviceToHost, st));
  JZ_CUDA(cudaStreamSynchronize(st));
  int ip = 0;
  for (int i = 1; i < n0; ++i)
    if (std::fabs(xs[i] - x) < std::fabs(xs[ip] - x)) ip = i;
  const size_t m = (size_t)n1 * n2;
  // a cylinder's last azimuthal plane repeats its first: not binned twice
  const size_t mb = s->g->dev.L.cyl ? (size_t)n1 * (size_t)s->g->dev.L.pn[2] : m;
  std::vector<double> yz(2 * m), su(m), su2(m);
  JZ_CUDA(launch_stats_plane_yz(s->g->dev, ip, s->scr, st));
  JZ_CUDA(cudaMemcpyAsync(yz.data(), s->scr, 16 * m, cudaMemcpyDeviceToHost, st));
  JZ_CUDA(cudaMemcpy2DAsync(su.data(), 8, s->su + ip, 8 * (size_t)n0, 8, m, cudaMemcpyDeviceToHost, st));
  JZ_CUDA(cudaMemcpy2DAsync(su2.data(), 8, s->su2 + ip, 8 * (size_t)n0, 8, m, cudaMemcpyDeviceToHost, st));
  JZ_CUDA(cudaStreamSynchronize(st));
  for (int b = 0; b < nbins; ++b) mean_u[b] = rms_u[b] = count[b] = 0.0;
  const double ns = (double)s->samples;
  for (size_t t = 0; t < mb; ++t) {  // nodes in [k][j] order
    const double r = std::sqrt(yz[2 * t] * yz[2 * t] + yz[2 * t + 1] * yz[2 * t + 1]);
    if (!(r < r_max)) continue;
    const int b = std::min(nbins - 1, (int)(r / r_max * nbins));
    const double mu = su[t] / ns;
    mean_u[b] += mu;
    rms_u[b] += std::sqrt(std::max(su2[t] / ns - mu * mu, 0.0));
    count[b] += 1.0;
  }
  for (int b = 0; b < nbins; ++b)
    if (count[b] > 0.0) {
      mean_u[b] /= count[b];
      rms_u[b] /= count[b];
    }
  return JZ_OK;
}

int jz_stats_core_length(jz_stats* s, double u_jet, double frac, double* length) {
  if (!s || !length) return fail(JZ_EINVAL, "null argument");
  if (!(u_jet > 0.0) || !(frac > 0.0)) return fail(JZ_EINVAL, "need u_jet > 0 and frac > 0");
  if (s->samples < 1) return fail(JZ_EINVAL, "no samples");
  const Layout& L = s->g->dev.L;
  const int n0 = L.n[0], n1 = L.n[1];
  cudaStream_t st = s->g->stream;
  // the node lines of the axis: on a box the one, two or four lines nearest
  // y = z = 0; on a cylinder the centreline j = 0 at its P distinct azimuths
  std::vector<std::pair<int, int>> lines;
  if (L.cyl) {
    for (int k = 0; k < L.pn[2]; ++k) lines.push_back({0, k});
  } else {
    int cj[2], ck[2], mj, mk;
    axis_nodes(L.n[1], cj, mj);
    axis_nodes(L.n[2], ck, mk);
    for (int a = 0; a < mj; ++a)
      for (int b = 0; b < mk; ++b) lines.push_back({cj[a], ck[b]});
  }
  std::vector<double> xs(n0), axis(n0, 0.0), line(n0);
  JZ_CUDA(launch_stats_axis_x(s->g->dev, lines[0].first, lines[0].second, s->scr, st));
  JZ_CUDA(cudaMemcpyAsync(xs.data(), s->scr, 8 * (size_t)n0, cudaMemcpyDeviceToHost, st));
  JZ_CUDA(cudaStreamSynchronize(st));
  // <U> on the axis: the mean over those lines
  for (const auto& jk : lines) {
    const size_t off = (size_t)n0 * (jk.first + (size_t)n1 * jk.second);
    JZ_CUDA(cudaMemcpyAsync(line.data(), s->su + off, 8 * (size_t)n0, cudaMemcpyDeviceToHost, st));
    JZ_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < n0; ++i) axis[i] += line[i];
  }
  const double level = frac * u_jet, ns = (double)s->samples * (double)lines.size();
  for (int i = 0; i < n0; ++i) axis[i] /= ns;
  // the first crossing below frac * u_jet from the inlet, interpolated linearly
  double len = xs[n0 - 1];
  if (axis[0] < level) len = xs[0];
  else
    for (int i = 1; i < n0; ++i)
      if (axis[i] < level) {
        len = xs[i - 1] + (xs[i] - xs[i - 1]) * (axis[i - 1] - level) / (axis[i - 1] - axis[i]);
        break;
      }
  *length = len;
  return JZ_OK;
}

int jz_stats_destroy(jz_stats* s) {
  delete s;
  return JZ_OK;
}

}  // extern "C"
