// api.cu -- libstag's C ABI: context, gauge-field upload, the operator calls
// and the mixed-precision CG driver (Sec. 3 of the paper: a mixed-precision
// CG inverter for staggered quarks, single precision dominant, with a double
// precision part).
//
// CG driver.  Per iteration, for every running system j (all on the GPU, no
// host round trip), two kernels:
//   K1  t = D_oe r + beta t_old (= D_oe p for p = r + beta p_old);
//       |t|^2, with |p|^2 = rho + 2 beta Re<r,p_old> + beta^2 |p_old|^2 ->
//       alpha = rho / (4 m_j^2 |p|^2 + |t|^2) (= <p, A p>, D_eo^dag = -D_oe)
//       (with FP16/BF16 Krylov vectors: p formed in the gather, |p|^2 reduced)
//   K2  p = r + beta p_old at the centre (stored); A p = 4 m^2 p - D_eo t;
//       r -= alpha A p; x_lo += alpha p; |r|^2, Re<r,p> -> beta; reliable-
//       update and convergence triggers                   (FP64 reduction)
//   Each kernel finishes the reduction of the one before it in every block
//   (fold), so a pass of SOLVE_UNROLL iterations ends with one finalize
//   kernel, which also sets the graph conditions.
//   if a reliable update is pending (a conditional graph node at the end of
//   every pass):
//   K4  x64 += x_lo,  x_lo = 0;  t = D_oe p (restarts the t recurrence)
//   K5  t64 = D_oe x64                                    (FP64)
//   K6  r = b - (4 m^2 x64 - D_eo t64) in FP64, stored at the residual's
//       precision; ||r||^2, Re<r,p> in FP64 -> true residual, convergence, beta
// The iterations sit in the body of a CUDA-graph WHILE node whose condition
// the pass's finalize / K6's finalize sets ("any system still running"); the
// update kernels sit in an IF node set by the pass's finalize.  One graph
// launch runs the whole solve.
// Without conditional-node support the same kernel sequence runs eagerly, with
// the host polling a device flag every few loop passes.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "launch.h"
#include "stag.h"

using namespace stag;

namespace {

size_t cplx_bytes(int P) { return P == P64 ? 16 : P == P32 ? 8 : 4; }

struct DevBuf {
  void *p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { reset(); }
  void reset() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n && p) return cudaSuccess;
    reset();
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    n = bytes;
    return cudaSuccess;
  }
};

// a set of nsys checkerboard vectors at one storage precision: its own
// allocation (ensure) or a view into a shared pool (set_view)
struct VecBuf {
  DevBuf data, scale;
  void *vdata = nullptr;   // view: data and scale inside another buffer (not owned)
  float *vscale = nullptr;
  size_t vbytes = 0;
  int prec = -1, nsys = 0, Ve = 0;
  void set_view(int P, int ns, int ve, void *d, float *sc, size_t bytes) {
    vdata = d;
    vscale = sc;
    vbytes = bytes;
    prec = P;
    nsys = ns;
    Ve = ve;
  }
  void *dptr() const { return vdata ? vdata : data.p; }
  size_t dbytes() const { return vdata ? vbytes : data.n; }
  float *sptr() const { return vdata ? vscale : (float *)scale.p; }
  cudaError_t ensure(int P, int ns, int ve) {
    vdata = nullptr;
    vscale = nullptr;
    cudaError_t e = data.ensure(cplx_bytes(P) * 3ull * ns * ve);
    if (e != cudaSuccess) return e;
    if (P == P16 || P == PBF) {
      e = scale.ensure(sizeof(float) * (size_t)ns * ve);
      if (e != cudaSuccess) return e;
    }
    prec = P;
    nsys = ns;
    Ve = ve;
    return cudaSuccess;
  }
  VecArg arg() const {
    VecArg a;
    a.v = dptr();
    a.scale = sptr();
    a.sstr = 3ll * Ve;
    return a;
  }
};

struct PinnedBuf {
  void *p = nullptr;
  size_t n = 0;
  PinnedBuf() = default;
  PinnedBuf(const PinnedBuf &) = delete;
  PinnedBuf &operator=(const PinnedBuf &) = delete;
  ~PinnedBuf() {
    if (p) cudaFreeHost(p);
  }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n && p) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMallocHost(&p, bytes ? bytes : 16);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
};

// solver workspace for one (number of systems, precision, link format)
struct Work {
  int nsys = 0, prec = -1, recon = -1;
  int VP = P32;  // precision of the Krylov vectors p and t
  int RP = P32;  // precision of the iterated residual r and partial solution x_lo
  int NS = 1, G = 1, NS64 = 1, G64 = 1;
  int lanes = 1, lanes64 = 1;  // lanes per site of the inner / FP64 half operator (tuned)
  int lanes_k1 = 1, lanes_k2 = 1;  // lanes of the two CG kernels (tuned with their epilogues)
  int nbx_k1 = 0, nbx_k2 = 0;      // blocks per system group of the two CG kernels
  int tma = 0;                     // link path of the CG kernels (DsArgs::tma)
  int l2p = 0;                     // L2 persistence during a solve: 1 the links, 2 the Krylov vectors
  int mrhs = 0;                    // > 0: the CG kernels are k_dslash_mrhs with mrhs systems per block
  int ms = 0;                      // > 0: multi-shift CG, ms shifted systems ride on each system
  int nrhs_sl = 0;                 // > 0: the CG kernels are k_cg_nrhs (every system in every block,
                                   // the links staged once per tile): threads per site, + 10 with
                                   // one link stage
  const void *links_tile = nullptr;
  int nbx_bl = 0, pstride = 0;
  VecBuf b64, x64, t64, r, x, p, t;
  DevBuf vpool;  // r, x, p, t (and their scales) in one range: one L2 window can cover them
  DevBuf st, partials, tickets, flags;
  DevBuf st2, partials2;  // second buffers of the states and partials (folded reductions)
  PinnedBuf h_st, h_flags;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_tried = false;
  cudaGraphConditionalHandle h_loop = 0, h_update = 0;
  unsigned long long gen = 0;  // bumped whenever captured kernels may hold stale arguments
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    graph_tried = false;
    ++gen;
  }
  ~Work() { drop_graph(); }
};

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct stag_ctx {
  int dims[4];
  int flags;
  int device;
  cudaStream_t stream;
  cudaStream_t cap = nullptr, cap2 = nullptr;  // private streams used only for graph capture
  Geom g;
  long long V;
  int Ve;
  std::string err;
  bool have_links = false;
  bool use_graph = true;
  bool pdl = true;  // CG kernels launched as programmatic dependents of their predecessors
  bool fold = true;     // each CG kernel finishes its predecessor's reduction itself
  bool persist = true;  // CG kernels launched as one wave of resident blocks
  int tma_modes = 0b101;  // link paths (bit t: DsArgs::tma = t) the tuner may choose for one system
  // STAG_TEST_WAIT_GIVEUP=1: in the solve loop, the bounded waits of the
  // shared-memory link path give up at once (tests of the failure path)
  int wait_giveup = 0;
  // L2 residency of the inner-precision links during a solve: the CG kernels
  // mark them as an access-policy window whose lines persist in L2 (the rest
  // of their traffic streams), so of the two passes over the links per
  // iteration most hit L2; the persisting lines are released after the solve
  bool l2persist = true;  // the device supports it and it is not switched off
  int l2_modes = 0b11;    // 0b11: by rule; else bit p: the tuner may choose L2 mode p (STAG_L2PERSIST fixes it)
  size_t l2_max_persist = 0, l2_max_window = 0;
  DevBuf links_canon;  // [4][V][3][3] FP64, kept for lazy reduced-precision copies
  DevBuf links64;
  DevBuf links_lo[4][2];
  bool lo_ok[4][2] = {{false, false}, {false, false}, {false, false}, {false, false}};
  DevBuf links_tile[4][2];  // tiled site-owned copies (bulk-copied by the CG kernels)
  bool tile_ok[4][2] = {{false, false}, {false, false}, {false, false}, {false, false}};
  DevBuf stage_in, stage_out;  // FP64 ABI-layout vectors for host transfers
  VecBuf api_a, api_b, api_c;  // internal vectors of the operator calls
  VecBuf full_e, full_o, full_x;  // full-lattice solve: halves of the sources, odd half of a solution
  DevBuf red;                     // block sums of the action's reduction
  DevBuf hyp_b, hyp_t, hyp_io;    // HYP smearing: the two decorated levels, host staging
  DevBuf npr_f, npr_o;            // NPR contraction: staged fields, per-hypercube values and their sum
  VecBuf ms_p, ms_x;              // multi-shift CG: shifted directions and solutions (FP32)
  DevBuf ms_sh;                   // their ShiftState
  PinnedBuf ms_h;
  DevBuf defect;
  Work w;
  int last_nsys = 0;  // systems of the most recent solve (stats in w.h_st)
  unsigned long long id = 0;  // process-unique, never reused
};

namespace {

int fail(stag_ctx *c, int code, const char *what, cudaError_t e) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  c->err = buf;
  cudaGetLastError();
  return code;
}

int arg_err(stag_ctx *c, const char *msg) {
  if (c) c->err = msg;
  return STAG_ERR_ARG;
}

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(c, e_ == cudaErrorMemoryAllocation ? STAG_ERR_OOM : STAG_ERR_CUDA, #call, e_); \
  } while (0)

#define CKS(expr)            \
  do {                       \
    int s_ = (expr);         \
    if (s_ != STAG_OK) return s_; \
  } while (0)

int valid_prec(int p) { return p == P64 || p == P32 || p == P16 || p == PBF; }

// Solver precision argument: link storage in the low byte; the Krylov vectors
// p and t at FP32, or at FP16/BF16 (per-site scaled) with STAG_VEC_FP16 /
// STAG_VEC_BF16 (any reduced-precision links) or STAG_HALF_VECTORS (the
// links' own FP16/BF16).  The residual and the partial solution stay FP32.
bool solver_precs(int precision, int *LP, int *VP, int *RP) {
  const int P = precision & 0xff;
  const int vbits = precision & (STAG_HALF_VECTORS | STAG_VEC_FP16 | STAG_VEC_BF16);
  if (!valid_prec(P) || (precision & ~(0xff | STAG_HALF_VECTORS | STAG_VEC_FP16 | STAG_VEC_BF16))) return false;
  int vp = (P == P64) ? P64 : P32;
  if (vbits == STAG_HALF_VECTORS) {
    if (!(P == P16 || P == PBF)) return false;
    vp = P;
  } else if (vbits == STAG_VEC_FP16 || vbits == STAG_VEC_BF16) {
    const int want = (vbits == STAG_VEC_FP16) ? P16 : PBF;
    // FP32 links with either; half links with vectors of their own format
    if (!(P == P32 || P == want)) return false;
    vp = want;
  } else if (vbits != 0) {
    return false;  // more than one vector format
  }
  *LP = P;
  *VP = vp;
  *RP = (P == P64) ? P64 : P32;
  return true;
}

// device pointer to the FP64 ABI vector `src` (copied through `stage` when on the host)
int vec_in(stag_ctx *c, const double *src, DevBuf &stage, size_t off_bytes, const double2 **out) {
  const size_t bytes = sizeof(double) * 6ull * c->Ve;
  if (is_device_ptr(src)) {
    *out = reinterpret_cast<const double2 *>(src);
    return STAG_OK;
  }
  CK(stage.ensure(off_bytes + bytes));
  CK(cudaMemcpyAsync((char *)stage.p + off_bytes, src, bytes, cudaMemcpyHostToDevice, c->stream));
  *out = reinterpret_cast<const double2 *>((char *)stage.p + off_bytes);
  return STAG_OK;
}

// write internal vector k of `v` (precision v.prec) to the FP64 ABI buffer dst
int vec_out(stag_ctx *c, const VecBuf &v, int k, double *dst) {
  const size_t bytes = sizeof(double) * 6ull * c->Ve;
  if (is_device_ptr(dst)) {
    CK(launch_unpack_vec(v.prec, v.arg(), k, reinterpret_cast<double2 *>(dst), c->Ve, c->stream));
    return STAG_OK;
  }
  CK(c->stage_out.ensure(bytes));
  CK(launch_unpack_vec(v.prec, v.arg(), k, reinterpret_cast<double2 *>(c->stage_out.p), c->Ve, c->stream));
  CK(cudaMemcpyAsync(dst, c->stage_out.p, bytes, cudaMemcpyDeviceToHost, c->stream));
  return STAG_OK;
}

int links_for(stag_ctx *c, int P, const void **out) {
  if (!c->have_links) {
    c->err = "no gauge field: call stag_links_upload first";
    return STAG_ERR_STATE;
  }
  if (P == P64) {
    *out = c->links64.p;
    return STAG_OK;
  }
  const int rc = (c->flags & STAG_RECON12) ? 1 : 0;
  if (!c->lo_ok[P][rc]) {
    const size_t ne = rc ? 6 : 9;
    CK(c->links_lo[P][rc].ensure(cplx_bytes(P) * ne * 8ull * c->Ve));
    CK(launch_pack_links(P, rc, reinterpret_cast<const double2 *>(c->links_canon.p), c->links_lo[P][rc].p,
                         c->g, c->stream));
    c->lo_ok[P][rc] = true;
  }
  *out = c->links_lo[P][rc].p;
  return STAG_OK;
}

// the tiled site-owned links at precision P (P32, P16 or PBF), built on first use
int links_tile_for(stag_ctx *c, int P, const void **out) {
  if (!c->have_links) {
    c->err = "no gauge field: call stag_links_upload first";
    return STAG_ERR_STATE;
  }
  const int rc = (c->flags & STAG_RECON12) ? 1 : 0;
  if (!c->tile_ok[P][rc]) {
    const size_t ne = rc ? 6 : 9;
    const size_t bytes = cplx_bytes(P) * ne * 8ull * LT * 2ull * (size_t)link_tiles(c->Ve);
    CK(c->links_tile[P][rc].ensure(bytes));
    CK(cudaMemsetAsync(c->links_tile[P][rc].p, 0, bytes, c->stream));
    CK(launch_pack_links_tiled(P, rc, reinterpret_cast<const double2 *>(c->links_canon.p), c->links_tile[P][rc].p,
                               c->g, link_tiles(c->Ve), c->stream));
    c->tile_ok[P][rc] = true;
  }
  *out = c->links_tile[P][rc].p;
  return STAG_OK;
}

// The L2 set-aside for persisting lines, held only while work that marks links
// persisting runs: set aside and unused, it still cost 16-source solves (which
// never mark anything persisting) most of their L2 hits.
void l2_setaside(stag_ctx *c, bool on) {
  if (!c->l2persist) return;
  // persisting vectors need only their own size set aside; the rest of L2 stays
  // with the streaming links
  size_t want = c->l2_max_persist;
  if (c->w.l2p == 2 && c->w.vpool.n < want) want = c->w.vpool.n;
  cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, on ? want : 0);
  cudaGetLastError();
}

// the L2 window of the CG kernels: on = 1 their links (link path tma,
// DsArgs::tma), on = 2 the Krylov vectors r, x, p, t of the workspace
void set_l2_window(stag_ctx *c, int P, int tma, int on, DsArgs &a) {
  a.l2_base = nullptr;
  a.l2_bytes = 0;
  a.l2_hit = 0.f;
  if (!c->l2persist || !on) return;
  const int rc = (P != P64 && (c->flags & STAG_RECON12)) ? 1 : 0;
  const DevBuf &b = (on == 2) ? c->w.vpool
                              : (P == P64) ? c->links64 : (tma ? c->links_tile[P][rc] : c->links_lo[P][rc]);
  if (!b.p || b.n == 0) return;
  a.l2_base = b.p;
  a.l2_bytes = b.n < c->l2_max_window ? b.n : c->l2_max_window;
  const double h = (double)c->l2_max_persist / (double)a.l2_bytes;
  a.l2_hit = h < 1.0 ? (float)h : 1.f;
}

int link_recon(const stag_ctx *c, int P) { return (P != P64 && (c->flags & STAG_RECON12)) ? 1 : 0; }

Ctl no_ctl() {
  Ctl k;
  memset(&k, 0, sizeof k);
  return k;
}

// ---------------------------------------------------------------------------
// autotuner: lanes per output site of the half operator
// ---------------------------------------------------------------------------
// The choice (1 or 2 lanes per site) is made per (link precision, reconstruct,
// vector precision, systems per thread, system groups, lattice) by timing the
// candidates with CUDA events (the plain operator: 3 warm-up and 10 timed
// launches on the caller's buffers; the CG kernels: tune_cg_pair) and is
// cached for the process.  STAG_LANES
// = 1 or 2 forces a value; STAG_TUNE_CACHE names a text file that persists the
// cache ("key lanes" lines) across processes.
typedef std::tuple<int, int, int, int, int, int, int, int, int> TuneKey;
std::map<TuneKey, int> g_tune;
std::mutex g_tune_mu;
bool g_tune_loaded = false;

std::string tune_key_str(const TuneKey &k) {
  char b[160];
  snprintf(b, sizeof b, "%d_%d_%d_%d_%d_%dx%dx%dx%d", std::get<0>(k), std::get<1>(k), std::get<2>(k),
           std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k), std::get<7>(k), std::get<8>(k));
  return b;
}

void tune_cache_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = getenv("STAG_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  int v[9], lanes;
  while (fscanf(f, "%d_%d_%d_%d_%d_%dx%dx%dx%d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &v[7],
                &v[8], &lanes) == 10)
    g_tune[TuneKey(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8])] = lanes;
  fclose(f);
}

void tune_cache_store(const TuneKey &k, int lanes) {
  const char *path = getenv("STAG_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d\n", tune_key_str(k).c_str(), lanes);
  fclose(f);
}

// Time both mappings of one instantiation: `a` holds the kernel's arguments.
// Blocks per system group of a CG kernel with `lanes` lanes per site: one
// wave of resident blocks over all groups (the kernel strides over its
// chunks of sites), at most one block per chunk.
int cg_blocks(stag_ctx *c, int LP, int recon, int VP, int NS, int EPI, int lanes, int G, int tma, int *nbx) {
  const int full = ds_blocks(c->Ve, lanes);
  *nbx = full;
  if (!c->persist) return STAG_OK;
  DsArgs none;
  memset(&none, 0, sizeof none);
  none.tma = tma;
  const void *k = nullptr;
  CK(launch_dslash(LP, recon, VP, VP, NS, EPI, lanes, 0, c->stream, none, &k));
  int per_sm = 0, nsm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, DS_BT, tma == 1 ? tma_smem_bytes(LP, recon, lanes) : 0));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  int n = per_sm * nsm / G;
  if (n < 1) n = 1;
  if (n < full) *nbx = n;
  return STAG_OK;
}

// The launch form of the two CG kernels, chosen together: lanes per site of
// each (1 or 2) and, where allowed (tma_ok: one system, reduced-precision
// links), the link path of both (DsArgs::tma, among c->tma_modes); whether
// their links persist in L2 follows a rule (below).  Each candidate
// runs tune_pairs() alternating launch pairs with the solver's grids, twice (the second
// sweep in reverse order), and the fastest total wins: the iteration
// alternates the two kernels, each starting on the cache state the other
// leaves.  Cached as 1000 l2p + 100 tma + 10 l1 + l2.  STAG_LANES = 1 or 2
// fixes the lanes.
// alternating launch pairs per timed sweep of the tuner: 20 at 20^3 x 64 and
// below, fewer on larger lattices (at least 3), so that tuning stays well under
// a second of kernel time
int tune_pairs(const stag_ctx *c) {
  const double n = 20.0 * 256000.0 / (double)c->Ve;
  return n >= 20.0 ? 20 : n <= 3.0 ? 3 : (int)n;
}

// Blocks per system group of k_dslash_mrhs with nsw systems per block: one
// wave of resident blocks, at most one per 32-site chunk.
int mrhs_blocks(stag_ctx *c, int recon, int nsw, int EPI, int G, int *nbx) {
  const int full = (c->Ve + 31) / 32;
  *nbx = full;
  if (!c->persist) return STAG_OK;
  DsArgs none;
  memset(&none, 0, sizeof none);
  const void *k = nullptr;
  CK(launch_dslash_mrhs(P32, recon, nsw, EPI, 0, c->stream, none, &k));
  int per_sm = 0, nsm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * nsw, 0));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  int n = per_sm * nsm / G;
  if (n < 1) n = 1;
  if (n < full) *nbx = n;
  return STAG_OK;
}

// total time of 2 sweeps of tune_pairs() alternating launch pairs of the two
// k_dslash_mrhs CG kernels with nsw systems per block (the measure
// tune_cg_pair reports)
int time_mrhs_pair(stag_ctx *c, int recon, int nsw, DsArgs a1, DsArgs a2, float *ms_out) {
  const int G = (a1.nsys + nsw - 1) / nsw;
  a1.ngroups = a2.ngroups = G;
  int n1 = 0, n2 = 0;
  CKS(mrhs_blocks(c, recon, nsw, EPI_CG_K1R, G, &n1));
  CKS(mrhs_blocks(c, recon, nsw, EPI_CG_K2, G, &n2));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float tot = 0.f;
  const int np = tune_pairs(c);
  for (int o = 0; o < 2; ++o) {
    for (int i = 0; i < np + 2; ++i) {
      if (i == 2) CK(cudaEventRecord(e0, c->stream));
      CK(launch_dslash_mrhs(P32, recon, nsw, EPI_CG_K1R, n1 * G, c->stream, a1));
      CK(launch_dslash_mrhs(P32, recon, nsw, EPI_CG_K2, n2 * G, c->stream, a2));
    }
    CK(cudaEventRecord(e1, c->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    tot += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = tot;
  return STAG_OK;
}

// Blocks of k_cg_nrhs with sl threads per site: one wave of resident
// blocks, at most one per tile of LT sites.
int nrhs_blocks(stag_ctx *c, int recon, int sl, int EPI, int *nb) {
  const int full = (c->Ve + LT - 1) / LT;
  DsArgs none;
  memset(&none, 0, sizeof none);
  const void *k = nullptr;
  CK(launch_cg_nrhs(recon, sl, EPI, 0, c->stream, none, &k));
  int per_sm = 0, nsm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, LT * (sl % 10),
                                                   cg_nrhs_smem(recon, nrhs_kernel_form(sl, EPI))));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  int n = per_sm * nsm;
  if (n < 1) n = 1;
  *nb = n < full ? n : full;
  return STAG_OK;
}

// total time of 2 sweeps of tune_pairs() alternating launch pairs of the two
// k_cg_nrhs kernels (the measure tune_cg_pair reports; no finalize between)
int time_nrhs_pair(stag_ctx *c, int recon, int sl, DsArgs a1, DsArgs a2, float *ms_out) {
  int n1 = 0, n2 = 0;
  CKS(nrhs_blocks(c, recon, sl, EPI_CG_K1R, &n1));
  CKS(nrhs_blocks(c, recon, sl, EPI_CG_K2, &n2));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float tot = 0.f;
  const int np = tune_pairs(c);
  for (int o = 0; o < 2; ++o) {
    for (int i = 0; i < np + 2; ++i) {
      if (i == 2) CK(cudaEventRecord(e0, c->stream));
      CK(launch_cg_nrhs(recon, sl, EPI_CG_K1R, n1, c->stream, a1));
      CK(launch_cg_nrhs(recon, sl, EPI_CG_K2, n2, c->stream, a2));
    }
    CK(cudaEventRecord(e1, c->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    tot += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = tot;
  return STAG_OK;
}

struct CgForm {
  int tma = 0, l1 = 1, l2 = 1, l2p = 0;  // link path, lanes of the two kernels, L2-persisting links
};

int tune_cg_pair(stag_ctx *c, int LP, int recon, int VP, int NS, int EPI1, DsArgs a1, DsArgs a2, bool tma_ok,
                 CgForm *out, float *ms_out = nullptr) {
  if (ms_out) *ms_out = -1.f;
  const int modes = tma_ok ? c->tma_modes : 1;  // bit t: link path t allowed
  // persisting links (bit p of l2modes: p allowed): by rule, not by timing --
  // short timings favoured them where whole solves ran slower.  On for one
  // system whose links fit the persisting set-aside to within 25 % (20^3 x 64
  // reconstruct-12 FP32: 98 MB against 84.7 MB, 10 % faster solves); off where
  // they do not fit (full FP32 links, 147 MB: 6 % slower) and for several
  // systems, whose vectors need the rest of L2 (16 sources: 27 % slower).
  int l2modes = 1;
  if (c->l2persist) {
    if (c->l2_modes != 0b11) {
      l2modes = c->l2_modes;
    } else {
      const int rc = (LP != P64 && recon) ? 1 : 0;
      const double lb = (double)cplx_bytes(LP) * (rc ? 6 : 9) * 8.0 * c->Ve;
      l2modes = (a1.nsys == 1 && lb <= 1.25 * (double)c->l2_max_persist) ? 0b10 : 0b01;
    }
  }
  // STAG_LANES = 1 or 2 fixes the lanes of both kernels; two digits (12, 21
  // ...) those of the first and the second
  const char *force = getenv("STAG_LANES");
  int fl1 = 0, fl2 = 0;
  if (force && (force[0] == '1' || force[0] == '2')) {
    if (force[1] == 0) fl1 = fl2 = force[0] - '0';
    else if ((force[1] == '1' || force[1] == '2') && force[2] == 0) fl1 = force[0] - '0', fl2 = force[1] - '0';
  }
  const bool fl = fl1 != 0;
  std::vector<CgForm> cand;
  for (int p = 0; p < 3; ++p)
    for (int t = 0; t < 3; ++t)
      for (int l1 = 1; l1 <= 2; ++l1)
        for (int l2 = 1; l2 <= 2; ++l2)
          if ((l2modes >> p & 1) && (modes >> t & 1) && (!fl || (l1 == fl1 && l2 == fl2))) {
            CgForm f;
            f.tma = t;
            f.l1 = l1;
            f.l2 = l2;
            f.l2p = p;
            cand.push_back(f);
          }
  if (cand.size() == 1 && !ms_out) {
    *out = cand[0];
    return STAG_OK;
  }
  const int G = a1.ngroups;
  const TuneKey key(LP, recon, VP, NS * 16 + EPI1 + 8, (G * 8 + modes) * 8 + l2modes, c->dims[0], c->dims[1],
                    c->dims[2], c->dims[3]);
  if (!fl && !ms_out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      out->l2p = it->second / 1000;
      out->tma = (it->second / 100) % 10;
      out->l1 = (it->second / 10) % 10;
      out->l2 = it->second % 10;
      return STAG_OK;
    }
  }
  const int nc = (int)cand.size();
  std::vector<int> nb1(nc), nb2(nc);
  for (int q = 0; q < nc; ++q) {
    int n = 0;
    CKS(cg_blocks(c, LP, recon, VP, NS, EPI1, cand[q].l1, G, cand[q].tma, &n));
    nb1[q] = n * G;
    CKS(cg_blocks(c, LP, recon, VP, NS, EPI_CG_K2, cand[q].l2, G, cand[q].tma, &n));
    nb2[q] = n * G;
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::vector<float> tot(nc, 0.f);
  for (int o = 0; o < 2 * nc; ++o) {
    const int q = o < nc ? o : 2 * nc - 1 - o;
    const CgForm &f = cand[q];
    a1.tma = a2.tma = f.tma;
    set_l2_window(c, LP, f.tma, f.l2p, a1);
    set_l2_window(c, LP, f.tma, f.l2p, a2);
    if (f.l2p) l2_setaside(c, true);
    for (int i = 0; i < tune_pairs(c) + 2; ++i) {
      if (i == 2) CK(cudaEventRecord(e0, c->stream));
      CK(launch_dslash(LP, recon, VP, VP, NS, EPI1, f.l1, nb1[q], c->stream, a1));
      CK(launch_dslash(LP, recon, VP, VP, NS, EPI_CG_K2, f.l2, nb2[q], c->stream, a2));
    }
    CK(cudaEventRecord(e1, c->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    tot[q] += ms;
    // each candidate starts without persisting lines
    if (f.l2p) {
      cudaCtxResetPersistingL2Cache();
      l2_setaside(c, false);
    }
    cudaGetLastError();
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int best = 0;
  for (int q = 1; q < nc; ++q)
    if (tot[q] < tot[best]) best = q;
  *out = cand[best];
  if (ms_out) *ms_out = tot[best];
  if (!fl) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int v = 1000 * out->l2p + 100 * out->tma + 10 * out->l1 + out->l2;
    g_tune[key] = v;
    tune_cache_store(key, v);
  }
  return STAG_OK;
}

int tune_lanes(stag_ctx *c, int LP, int recon, int VP, int NS, int G, int nsys, const void *links, VecArg in,
               VecArg out, int *lanes_out) {
  const char *force = getenv("STAG_LANES");
  if (force && (force[0] == '1' || force[0] == '2') && force[1] == 0) {
    *lanes_out = force[0] - '0';
    return STAG_OK;
  }
  const TuneKey key(LP, recon, VP, NS, G, c->dims[0], c->dims[1], c->dims[2], c->dims[3]);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      *lanes_out = it->second;
      return STAG_OK;
    }
  }
  DsArgs a;
  memset(&a, 0, sizeof a);
  a.g = c->g;
  a.links = links;
  a.in = in;
  a.out = out;
  a.nsys = nsys;
  a.ngroups = G;
  a.gate = GATE_NONE;
  a.fin = FIN_NONE;
  a.par_out = 1;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_l = 1;
  for (int l = 1; l <= 2; ++l) {
    const int nb = ds_blocks(c->Ve, l) * G;
    for (int i = 0; i < 3; ++i) CK(launch_dslash(LP, recon, VP, VP, NS, EPI_PLAIN, l, nb, c->stream, a));
    CK(cudaEventRecord(e0, c->stream));
    for (int i = 0; i < 10; ++i) CK(launch_dslash(LP, recon, VP, VP, NS, EPI_PLAIN, l, nb, c->stream, a));
    CK(cudaEventRecord(e1, c->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      best_l = l;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best_l;
    tune_cache_store(key, best_l);
  }
  *lanes_out = best_l;
  return STAG_OK;
}

// ---------------------------------------------------------------------------
// solver
// ---------------------------------------------------------------------------

Ctl work_ctl(stag_ctx *c, bool graph);
DsArgs ds_base(stag_ctx *c);

int work_prepare(stag_ctx *c, int nsys, int precision, int ms = 0) {
  Work &w = c->w;
  int prec, VP, RP;
  if (!solver_precs(precision, &prec, &VP, &RP)) return arg_err(c, "bad solver precision");
  const int recon = link_recon(c, prec);
  if (w.ms != ms) {  // the shift kernel enters or leaves the graph's loop body
    w.drop_graph();
    w.ms = ms;
  }
  if (w.nsys == nsys && w.prec == prec && w.VP == VP && w.recon == recon) return STAG_OK;
  w.drop_graph();
  c->last_nsys = 0;
  w.nsys = nsys;
  w.prec = prec;
  w.recon = recon;
  w.VP = VP;
  w.RP = RP;
  w.NS = 1;
  w.G = nsys;
  w.NS64 = nsys >= 4 ? 4 : 1;
  w.G64 = (nsys + w.NS64 - 1) / w.NS64;
  const int Ve = c->Ve;
  const int nbx_ds_max = (Ve + 31) / 32;  // most blocks per group of any CG kernel (32-site chunks)
  w.nbx_bl = (Ve + BLAS_BT - 1) / BLAS_BT;
  w.pstride = nbx_ds_max > w.nbx_bl ? nbx_ds_max : w.nbx_bl;
  CK(w.b64.ensure(P64, nsys, Ve));
  CK(w.x64.ensure(P64, nsys, Ve));
  CK(w.t64.ensure(P64, nsys, Ve));
  {
    // r, x_lo (RP) and p, t (VP) with their scales, 256-byte aligned, in one pool
    const size_t rb = (cplx_bytes(w.RP) * 3ull * nsys * Ve + 255) & ~(size_t)255;
    const size_t vb = (cplx_bytes(VP) * 3ull * nsys * Ve + 255) & ~(size_t)255;
    const size_t sb = (VP == P16 || VP == PBF) ? ((sizeof(float) * (size_t)nsys * Ve + 255) & ~(size_t)255) : 0;
    CK(w.vpool.ensure(2 * rb + 2 * vb + 2 * sb));
    char *b = (char *)w.vpool.p;
    w.r.set_view(w.RP, nsys, Ve, b, nullptr, rb);
    w.x.set_view(w.RP, nsys, Ve, b + rb, nullptr, rb);
    w.p.set_view(VP, nsys, Ve, b + 2 * rb, sb ? (float *)(b + 2 * rb + 2 * vb) : nullptr, vb);
    w.t.set_view(VP, nsys, Ve, b + 2 * rb + vb, sb ? (float *)(b + 2 * rb + 2 * vb + sb) : nullptr, vb);
  }
  CK(w.st.ensure(sizeof(SysState) * nsys));
  CK(w.partials.ensure(sizeof(double) * (size_t)nsys * NVMAX * w.pstride));
  CK(w.st2.ensure(sizeof(SysState) * nsys));
  CK(w.partials2.ensure(sizeof(double) * (size_t)nsys * NVMAX * w.pstride));
  const size_t ntickets = 1;
  CK(w.tickets.ensure(sizeof(unsigned) * ntickets));
  CK(w.flags.ensure(sizeof(int) * 8));
  CK(w.h_st.ensure(sizeof(SysState) * nsys));
  CK(w.h_flags.ensure(sizeof(int) * 8));
  CK(cudaMemsetAsync(w.tickets.p, 0, sizeof(unsigned) * ntickets, c->stream));
  CK(cudaMemsetAsync(w.st.p, 0, sizeof(SysState) * nsys, c->stream));
  CK(cudaMemsetAsync(w.st2.p, 0, sizeof(SysState) * nsys, c->stream));
  // defined contents for the timing entry point before any solve
  CK(cudaMemsetAsync(w.vpool.p, 0, w.vpool.n, c->stream));  // r, x, p, t and scales
  CK(cudaMemsetAsync(w.x64.data.p, 0, w.x64.data.n, c->stream));
  const void *lo = nullptr;
  CKS(links_for(c, prec, &lo));
  {
    // the two CG kernels with their own epilogues (state zeroed: alpha = beta = 0)
    DsArgs a = ds_base(c);
    a.links = lo;
    a.nsys = nsys;
    a.ngroups = w.G;
    a.ctl = work_ctl(c, false);
    a.gate = GATE_NONE;
    a.fin = FIN_NONE;
    a.aux = w.r.arg();
    a.xlo = w.x.arg();
    const bool tma_ok = (w.NS == 1 && prec != P64 && c->tma_modes != 1);
    w.links_tile = nullptr;
    if (tma_ok) CKS(links_tile_for(c, prec, &w.links_tile));
    a.links_tile = w.links_tile;
    a.ntile = link_tiles(c->Ve);
    const bool rec = (VP == w.RP);
    const int epi1 = rec ? EPI_CG_K1R : EPI_CG_K1;
    DsArgs a2 = a;
    a.par_out = 1;
    a.in = rec ? w.r.arg() : w.p.arg();
    a.out = w.t.arg();
    a2.par_out = 0;
    a2.in = w.t.arg();
    a2.center = w.p.arg();
    // Systems per thread of the CG kernels.  NS = 1 gives every system its own
    // blocks; the blocks of one chunk (consecutive in the grid) run together and
    // share its links through L2.  NS = 4 or 8 holds the links in registers
    // for all the thread's systems, at the price of registers (occupancy).
    // Several systems: the candidates are timed (kernel pair, tune_cg_pair)
    // and the choice cached; STAG_NS = 1, 4 or 8 fixes it.
    std::vector<int> cands{1};
    if (nsys >= 4) cands.push_back(4);
    if (nsys >= 8 && prec != P64) cands.push_back(8);
    const char *fns = getenv("STAG_NS");
    if (fns && (fns[0] == '1' || fns[0] == '4' || fns[0] == '8') && fns[1] == 0) {
      const int f = fns[0] - '0';
      if (f <= nsys && !(f == 8 && prec == P64)) cands.assign(1, f);
    }
    // the shared-memory kernels (k_dslash_mrhs): FP32 links and vectors, 4 or 8
    // systems per block; encoded as 100 + nsw among the candidates
    if (prec == P32 && VP == P32 && !(fns && fns[0] != 0)) {
      if (nsys >= 4) cands.push_back(104);
      if (nsys >= 8) cands.push_back(108);
    }
    const char *fmr = getenv("STAG_MRHS");
    if (fmr && (fmr[0] == '4' || fmr[0] == '8') && fmr[1] == 0 && prec == P32 && VP == P32 && nsys >= 2)
      cands.assign(1, 100 + (fmr[0] - '0'));
    // k_cg_nrhs (every system in every block, the links staged once per tile in
    // shared memory): FP32 links and vectors, 2..64 systems; encoded 200 + sl
    const bool nrhs_ok = prec == P32 && VP == P32 && nsys >= 2 && nsys <= CG_NRHS_MAX;
    if (nrhs_ok && !(fns && fns[0] != 0) && !(fmr && fmr[0] != 0)) {
      cands.push_back(202);
      cands.push_back(204);
      if (recon) cands.push_back(224);
    }
    // STAG_NRHS = 2 or 4: this form with that many threads per site (two link
    // stages), 14: 4 threads per site with one stage (3 blocks per SM; measured
    // slower: 48-system 20^3 x 64 solve 3.34 s vs 2.36 s, so not a default
    // candidate), 24: kernel 1 with two systems per pass through the thread
    // (reconstruct-12 links; kernel 2 as form 4); 0: never this form
    const char *fnr = getenv("STAG_NRHS");
    if (fnr && nrhs_ok) {
      const int f = atoi(fnr);
      if (f == 2 || f == 4 || f == 14 || (f == 24 && recon)) cands.assign(1, 200 + f);
    }
    if (fnr && fnr[0] == '0' && fnr[1] == 0) {
      std::vector<int> keep;
      for (int v : cands)
        if (v < 200) keep.push_back(v);
      cands = keep;
    }
    const void *tiled = nullptr;
    for (int v : cands)
      if (v > 200) {
        CKS(links_tile_for(c, prec, &tiled));
        a.links_tile = a2.links_tile = tiled;
        break;
      }
    int best_ns = cands[0];
    if (cands.size() > 1) {
      const TuneKey nkey(prec, recon, VP, 2000 + nsys, tma_ok ? 1 : 0, c->dims[0], c->dims[1], c->dims[2],
                         c->dims[3]);
      bool cached = false;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_load();
        auto it = g_tune.find(nkey);
        if (it != g_tune.end()) {
          best_ns = it->second;
          cached = true;
        }
      }
      if (!cached) {
        float best_ms = 1e30f;
        for (int ns : cands) {
          float ms = -1.f;
          if (ns > 200) {
            CKS(time_nrhs_pair(c, recon, ns - 200, a, a2, &ms));
          } else if (ns > 100) {
            CKS(time_mrhs_pair(c, recon, ns - 100, a, a2, &ms));
          } else {
            a.ngroups = a2.ngroups = (nsys + ns - 1) / ns;
            CgForm f;
            CKS(tune_cg_pair(c, prec, recon, VP, ns, epi1, a, a2, tma_ok && ns == 1, &f, &ms));
          }
          if (ms >= 0.f && ms < best_ms) {
            best_ms = ms;
            best_ns = ns;
          }
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[nkey] = best_ns;
        tune_cache_store(nkey, best_ns);
      }
    }
    w.nrhs_sl = best_ns > 200 ? best_ns - 200 : 0;
    w.mrhs = (best_ns > 100 && best_ns < 200) ? best_ns - 100 : 0;
    w.NS = w.mrhs ? w.mrhs : (w.nrhs_sl ? 1 : best_ns);
    w.G = (nsys + w.NS - 1) / w.NS;
    a.ngroups = a2.ngroups = w.G;
    if (w.nrhs_sl) {
      // the BLAS and update kernels keep one system per group; the CG kernels
      // are one grid of nbx_k1 / nbx_k2 blocks, each a partial per system
      CKS(links_tile_for(c, prec, &w.links_tile));
      w.tma = 1;
      w.lanes_k1 = w.lanes_k2 = w.nrhs_sl % 10;
      w.l2p = 0;
      CKS(nrhs_blocks(c, recon, w.nrhs_sl, EPI_CG_K1R, &w.nbx_k1));
      CKS(nrhs_blocks(c, recon, w.nrhs_sl, EPI_CG_K2, &w.nbx_k2));
    } else if (w.mrhs) {
      w.tma = 0;
      w.lanes_k1 = w.lanes_k2 = 1;
      w.l2p = 0;
      CKS(mrhs_blocks(c, recon, w.mrhs, EPI_CG_K1R, w.G, &w.nbx_k1));
      CKS(mrhs_blocks(c, recon, w.mrhs, EPI_CG_K2, w.G, &w.nbx_k2));
    } else {
      CgForm form;
      CKS(tune_cg_pair(c, prec, recon, VP, w.NS, epi1, a, a2, tma_ok && w.NS == 1, &form));
      w.tma = form.tma;
      w.lanes_k1 = form.l1;
      w.lanes_k2 = form.l2;
      w.l2p = form.l2p;
      CKS(cg_blocks(c, prec, recon, VP, w.NS, epi1, w.lanes_k1, w.G, w.tma, &w.nbx_k1));
      CKS(cg_blocks(c, prec, recon, VP, w.NS, EPI_CG_K2, w.lanes_k2, w.G, w.tma, &w.nbx_k2));
    }
  }
  // the thread mapping of the plain inner and the FP64 half operators
  CKS(tune_lanes(c, prec, recon, VP, w.NS, w.G, nsys, lo, w.p.arg(), w.t.arg(), &w.lanes));
  CKS(tune_lanes(c, P64, 0, P64, w.NS64, w.G64, nsys, c->links64.p, w.x64.arg(), w.t64.arg(), &w.lanes64));
  return STAG_OK;
}

Ctl work_ctl(stag_ctx *c, bool graph) {
  Work &w = c->w;
  Ctl k;
  memset(&k, 0, sizeof k);
  k.st = (SysState *)w.st.p;
  k.partials = (double *)w.partials.p;
  k.all_ticket = (unsigned *)w.tickets.p;
  k.flags = (int *)w.flags.p;
  k.pstride = w.pstride;
  k.use_graph_cond = graph ? 1 : 0;
  k.h_loop = w.h_loop;
  k.h_update = w.h_update;
  return k;
}

DsArgs ds_base(stag_ctx *c) {
  DsArgs a;
  memset(&a, 0, sizeof a);
  a.g = c->g;
  return a;
}

BlasArgs blas_base(stag_ctx *c, const Ctl &ctl) {
  Work &w = c->w;
  BlasArgs b;
  memset(&b, 0, sizeof b);
  b.Ve = c->Ve;
  b.p = w.p.arg();
  b.r = w.r.arg();
  b.x = w.x.arg();
  b.b = w.b64.arg();
  b.x64 = w.x64.arg();
  b.t = w.t.arg();
  b.nsys = w.nsys;
  b.ngroups = w.G;
  b.ctl = ctl;
  return b;
}

// One of the two CG kernels (kernel 0: epi1 = EPI_CG_K1R or EPI_CG_K1;
// kernel 1: EPI_CG_K2) in the workspace's tuned launch form.
cudaError_t launch_cg(stag_ctx *c, int kernel, int epi, cudaStream_t s, const DsArgs &a) {
  Work &w = c->w;
  if (w.nrhs_sl)
    return launch_cg_nrhs(w.recon, w.nrhs_sl, epi, kernel == 0 ? w.nbx_k1 : w.nbx_k2, s, a);
  const int nb = (kernel == 0 ? w.nbx_k1 : w.nbx_k2) * w.G;
  if (w.mrhs) return launch_dslash_mrhs(w.prec, w.recon, w.mrhs, epi, nb, s, a);
  return launch_dslash(w.prec, w.recon, w.VP, w.VP, w.NS, epi, kernel == 0 ? w.lanes_k1 : w.lanes_k2, nb, s, a);
}

// The shifted-system update of a multi-shift solve (w.ms > 0), launched
// between the two CG kernels; `fold` as the second kernel's (the first
// kernel's sums in fold_partials over states ctl.st), or FIN_NONE with the
// states already finalized.
constexpr double MS_SHIFT_TOL = 1e-5;  // shifts stop below this estimated residual (under their FP32 floor)

int launch_ms(stag_ctx *c, cudaStream_t s, const DsArgs &k2) {
  Work &w = c->w;
  MsArgs m;
  memset(&m, 0, sizeof m);
  m.d = k2;
  m.nsh = w.ms;
  m.r = w.r.arg();
  m.ps = c->ms_p.arg();
  m.xs = c->ms_x.arg();
  m.sh = (ShiftState *)c->ms_sh.p;
  m.tol2 = MS_SHIFT_TOL * MS_SHIFT_TOL;
  // blocks per base system: enough to cover the SMs with the systems together
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  const int full = (c->Ve + 127) / 128;
  int nbx = (8 * nsm + w.nsys - 1) / w.nsys;
  m.nbx = nbx < full ? (nbx < 1 ? 1 : nbx) : full;
  CK(launch_shift_update(m, s));
  return STAG_OK;
}

// One CG iteration with a finalize kernel after each CG kernel (the form
// without folded reductions, STAG_FOLD=0): K1, its finalize, K2, its finalize.
int enqueue_main(stag_ctx *c, cudaStream_t s, const Ctl &ctl) {
  Work &w = c->w;
  const void *lo = nullptr;
  CKS(links_for(c, w.prec, &lo));
  DsArgs a = ds_base(c);
  a.links = lo;
  a.nsys = w.nsys;
  a.ngroups = w.G;
  a.ctl = ctl;
  a.gate = GATE_RUNNING;
  a.aux = w.r.arg();
  a.xlo = w.x.arg();
  a.pdl = c->pdl ? 1 : 0;
  if (w.tma) CKS(links_tile_for(c, w.prec, &w.links_tile));
  a.tma = w.tma;
  a.wait_giveup = c->wait_giveup;
  a.links_tile = w.links_tile;
  a.ntile = link_tiles(c->Ve);
  set_l2_window(c, w.prec, w.tma, w.l2p, a);
  // K1: t = D_oe (r + beta p_old); |t|^2 (and |p|^2) -> alpha
  a.par_out = 1;
  a.in = (w.VP == w.RP) ? w.r.arg() : w.p.arg();
  a.out = w.t.arg();
  const int nbx = w.nbx_k1;
  if (w.VP == w.RP) {
    // t = D_oe r + beta t_old: one gathered vector; |p|^2 from the scalar recurrence
    a.out = w.t.arg();
    a.fin = FIN_ALPHA_R;
    CK(launch_cg(c, 0, EPI_CG_K1R, s, a));
    CK(launch_finalize(ctl, FIN_ALPHA_R, nbx, 1, w.nsys, s, c->pdl));
  } else {
    // FP16/BF16 Krylov vectors: no t recurrence (its rounding would accumulate)
    a.fin = FIN_ALPHA;
    CK(launch_cg(c, 0, EPI_CG_K1, s, a));
    CK(launch_finalize(ctl, FIN_ALPHA, nbx, 2, w.nsys, s, c->pdl));
  }
  if (w.ms > 0) {
    DsArgs m = a;
    m.fold = FIN_NONE;
    CKS(launch_ms(c, s, m));
  }
  // K2: p = r + beta p_old; Ap = 4 m^2 p - D_eo t; r -= alpha Ap; x += alpha p; |r|^2
  a.par_out = 0;
  a.in = w.t.arg();
  a.center = w.p.arg();
  a.fin = FIN_NORM;
  const int nbx2 = w.nbx_k2;
  CK(launch_cg(c, 1, EPI_CG_K2, s, a));
  CK(launch_finalize(ctl, FIN_NORM, nbx2, 2, w.nsys, s, c->pdl));
  return STAG_OK;
}

// One pass of the solve loop: `unroll` iterations.  With folded
// reductions each CG kernel finishes its predecessor's reduction itself, so
// the pass launches 2 unroll CG kernels and a single finalize kernel
// (the last reduction, which also sets the loop and update conditions).  The
// states and the partials alternate between two buffers, as a block may still
// read the old ones while another writes the new; the pass starts and ends with
// the states in w.st.
int enqueue_pass(stag_ctx *c, cudaStream_t s, const Ctl &ctl, int unroll) {
  Work &w = c->w;
  // k_cg_nrhs does not fold its predecessor's sums (each block holds every
  // system): a finalize kernel follows each CG kernel
  if (!c->fold || w.nrhs_sl) {
    for (int u = 0; u < unroll; ++u) CKS(enqueue_main(c, s, ctl));
    return STAG_OK;
  }
  const void *lo = nullptr;
  CKS(links_for(c, w.prec, &lo));
  SysState *S[2] = {(SysState *)w.st.p, (SysState *)w.st2.p};
  double *PA = (double *)w.partials.p, *PB = (double *)w.partials2.p;
  const bool rec = (w.VP == w.RP);
  DsArgs a = ds_base(c);
  a.links = lo;
  a.nsys = w.nsys;
  a.ngroups = w.G;
  a.ctl = ctl;
  a.gate = GATE_RUNNING;
  a.fin = FIN_NONE;
  a.aux = w.r.arg();
  a.xlo = w.x.arg();
  a.pdl = c->pdl ? 1 : 0;
  if (w.tma) CKS(links_tile_for(c, w.prec, &w.links_tile));
  a.tma = w.tma;
  a.wait_giveup = c->wait_giveup;
  a.links_tile = w.links_tile;
  a.ntile = link_tiles(c->Ve);
  set_l2_window(c, w.prec, w.tma, w.l2p, a);
  int cur = 0;  // buffer of the current states
  for (int u = 0; u < unroll; ++u) {
    // K1: t = D_oe (r + beta p_old); |t|^2 (and |p|^2); folds the previous K2's norms
    a.par_out = 1;
    a.in = rec ? w.r.arg() : w.p.arg();
    a.out = w.t.arg();
    a.center = VecArg();
    a.ctl.st = S[cur];
    a.ctl.partials = PA;
    a.fold = (u == 0) ? FIN_NONE : FIN_NORM;
    a.fold_partials = PB;
    a.fold_nbx = w.nbx_k2;
    a.fold_nv = 2;
    a.st_out = S[1 - cur];
    CK(launch_cg(c, 0, rec ? EPI_CG_K1R : EPI_CG_K1, s, a));
    if (u > 0) cur = 1 - cur;
    // K2: p = r + beta p_old; r -= alpha (4 m^2 p - D_eo t); x += alpha p; folds K1's sums
    a.par_out = 0;
    a.in = w.t.arg();
    a.out = VecArg();
    a.center = w.p.arg();
    a.ctl.st = S[cur];
    a.ctl.partials = PB;
    a.fold = rec ? FIN_ALPHA_R : FIN_ALPHA;
    a.fold_partials = PA;
    a.fold_nbx = w.nbx_k1;
    a.fold_nv = rec ? 1 : 2;
    a.st_out = S[1 - cur];
    if (w.ms > 0) CKS(launch_ms(c, s, a));
    CK(launch_cg(c, 1, EPI_CG_K2, s, a));
    cur = 1 - cur;
  }
  Ctl f = ctl;
  f.partials = PB;
  CK(launch_finalize(f, FIN_NORM, w.nbx_k2, 2, w.nsys, s, c->pdl, S[cur] == S[0] ? nullptr : S[cur]));
  return STAG_OK;
}

// The reliable update (K4..K6 of the header comment; every kernel gated per
// system: only systems with an update due take part)
int enqueue_update(stag_ctx *c, cudaStream_t s, const Ctl &ctl) {
  Work &w = c->w;
  BlasArgs b = blas_base(c, ctl);
  b.gate = GATE_UPDATE;
  b.fin = FIN_NONE;
  CK(launch_accum_x(w.RP, w.NS, w.nbx_bl * w.G, s, b));
  if (w.VP == w.RP) {
    // restart the t recurrence from t = D_oe p exactly
    const void *lo = nullptr;
    CKS(links_for(c, w.prec, &lo));
    DsArgs q = ds_base(c);
    q.links = lo;
    q.nsys = w.nsys;
    q.ngroups = w.G;
    q.ctl = ctl;
    q.gate = GATE_UPDATE;
    q.fin = FIN_NONE;
    q.par_out = 1;
    q.in = w.p.arg();
    q.out = w.t.arg();
    CK(launch_dslash(w.prec, w.recon, w.VP, w.VP, w.NS, EPI_PLAIN, w.lanes, ds_blocks(c->Ve, w.lanes) * w.G, s,
                     q));
  }
  DsArgs a = ds_base(c);
  a.links = c->links64.p;
  a.nsys = w.nsys;
  a.ngroups = w.G64;
  a.ctl = ctl;
  a.gate = GATE_UPDATE;
  a.par_out = 1;
  a.in = w.x64.arg();
  a.out = w.t64.arg();
  a.fin = FIN_NONE;
  CK(launch_dslash(P64, 0, P64, P64, w.NS64, EPI_PLAIN, w.lanes64, ds_blocks(c->Ve, w.lanes64) * w.G64, s, a));
  a.par_out = 0;
  a.in = w.t64.arg();
  a.center = w.x64.arg();
  a.aux = w.b64.arg();
  a.out = w.r.arg();
  a.fin = FIN_RESID;
  if (w.VP == w.RP) a.dir = w.p.arg();  // Re<r_true, p> for the |p|^2 recurrence
  CK(launch_dslash(P64, 0, P64, w.RP, w.NS64, EPI_RESID, w.lanes64, ds_blocks(c->Ve, w.lanes64) * w.G64, s, a));
  CK(launch_finalize(ctl, FIN_RESID, ds_blocks(c->Ve, w.lanes64), 2, w.nsys, s));
  return STAG_OK;
}

// Iterations per pass of the solve loop: the body holds SOLVE_UNROLL copies of
// K1, K2, one finalize kernel and one conditional reliable update (a pending
// update waits for the end of the pass), which spreads the loop, finalize and
// conditional-node overhead.  Measured at 20^3 x 64: 4 -> 155.1 ms, 8 -> 152.4,
// 16 -> 150.5 (same 2958 iterations); a converged system's remaining
// iterations of its pass are gated launches of a few us each.
constexpr int SOLVE_UNROLL = 16;

// iterations per pass (STAG_UNROLL = 1..16 overrides SOLVE_UNROLL)
int solve_unroll() {
  const char *u = getenv("STAG_UNROLL");
  const int v = u ? atoi(u) : 0;
  return (v >= 1 && v <= 16) ? v : SOLVE_UNROLL;
}

int build_graph_inner(stag_ctx *c);

// Build the solve graph; on failure close any open capture and report.
int build_graph(stag_ctx *c) {
  const int st = build_graph_inner(c);
  if (st != STAG_OK) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t tmp = nullptr;
    if (c->cap2 && cudaStreamIsCapturing(c->cap2, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      cudaStreamEndCapture(c->cap2, &tmp);
    if (c->cap && cudaStreamIsCapturing(c->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      cudaStreamEndCapture(c->cap, &tmp);
    cudaGetLastError();
  }
  return st;
}

// Add one context's solve loop to graph g: a WHILE node (condition: any
// system still running) whose body holds SOLVE_UNROLL iterations and an IF
// node (condition: a reliable update pending) around the update kernels.
// The conditional handles are stored in the context's workspace, where the
// captured kernels read them.
int add_solve_loop(stag_ctx *c, cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, cudaGraphNode_t *out) {
  Work &w = c->w;
  if (!c->cap) CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  if (!c->cap2) CK(cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking));
  CK(cudaGraphConditionalHandleCreate(&w.h_loop, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp = {cudaGraphNodeTypeConditional};
  wp.conditional.handle = w.h_loop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wn;
  CK(cudaGraphAddNode(&wn, g, deps, nullptr, ndeps, &wp));
  if (out) *out = wn;
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  CK(cudaGraphConditionalHandleCreate(&w.h_update, body, 0, cudaGraphCondAssignDefault));
  const Ctl ctl = work_ctl(c, true);

  CK(cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int st = STAG_OK;
  st = enqueue_pass(c, c->cap, ctl, solve_unroll());
  if (st != STAG_OK) {
    cudaGraph_t tmp;
    cudaStreamEndCapture(c->cap, &tmp);
    return st;
  }
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t *cdeps = nullptr;
  size_t ncdeps = 0;
  cudaGraph_t capg = nullptr;
  CK(cudaStreamGetCaptureInfo(c->cap, &cs, nullptr, &capg, &cdeps, nullptr, &ncdeps));
  std::vector<cudaGraphNode_t> dv(cdeps, cdeps + ncdeps);
  cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
  ip.conditional.handle = w.h_update;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t ifn;
  CK(cudaGraphAddNode(&ifn, capg, dv.data(), nullptr, dv.size(), &ip));
  CK(cudaStreamUpdateCaptureDependencies(c->cap, &ifn, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(c->cap2, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  st = enqueue_update(c, c->cap2, ctl);
  {
    cudaGraph_t tmp;
    CK(cudaStreamEndCapture(c->cap2, &tmp));
  }
  if (st != STAG_OK) return st;
  {
    cudaGraph_t tmp;
    CK(cudaStreamEndCapture(c->cap, &tmp));
  }
  return STAG_OK;
}

int build_graph_inner(stag_ctx *c) {
  Work &w = c->w;
  w.graph_tried = true;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  w.graph = g;
  CKS(add_solve_loop(c, g, nullptr, 0, nullptr));
  CK(cudaGraphInstantiate(&w.exec, g, 0));
  return STAG_OK;
}

// Solve phases (shared by the single, the ragged and the full-lattice solve)
// start: per-system parameters and the CG start, on c->stream, with the
// sources already in w.b64.  full != nullptr (a full-lattice solve): the even
// and odd halves of the full sources, whose (2m)^2 |b|^2 becomes each
// system's reference norm.
struct FullRef {
  VecArg be, bo;
};
int solve_start(stag_ctx *c, const double masses[], int nmass, double tol, int maxiter, const FullRef *full);

// stage: sources, per-system parameters and the CG start, on c->stream
int solve_stage(stag_ctx *c, const double *const src[], int nrhs, const double masses[], int nmass, double tol,
                int maxiter, int prec) {
  const int nsys = nrhs * nmass;
  CKS(work_prepare(c, nsys, prec));
  Work &w = c->w;
  const void *lo = nullptr;
  CKS(links_for(c, w.prec, &lo));
  // sources -> b64 (FP64 internal layout)
  for (int r = 0; r < nrhs; ++r) {
    const double2 *d = nullptr;
    CKS(vec_in(c, src[r], c->stage_in, 0, &d));
    for (int k = 0; k < nmass; ++k) CK(launch_pack_vec(P64, d, w.b64.arg(), r * nmass + k, c->Ve, c->stream));
  }
  return solve_start(c, masses, nmass, tol, maxiter, nullptr);
}

int solve_start(stag_ctx *c, const double masses[], int nmass, double tol, int maxiter, const FullRef *full) {
  Work &w = c->w;
  const int nsys = w.nsys;
  // per-system parameters
  SysState *hs = (SysState *)w.h_st.p;
  CK(cudaStreamSynchronize(c->stream));  // pinned staging buffer reuse
  for (int j = 0; j < nsys; ++j) {
    memset(&hs[j], 0, sizeof(SysState));
    const double m = masses[j % nmass];
    hs[j].m4 = 4.0 * m * m;
    hs[j].tol = tol;
    hs[j].delta = (w.prec == P64) ? 0.0 : 0.1;
    hs[j].maxiter = maxiter;
    hs[j].ref_full = full ? 1 : 0;
  }
  CK(cudaMemcpyAsync(w.st.p, hs, sizeof(SysState) * nsys, cudaMemcpyHostToDevice, c->stream));
  {
    // loop-pass counter and its cap (an absolute bound on the solve loop)
    int *hf = (int *)w.h_flags.p;
    hf[0] = 1;
    hf[1] = 0;
    hf[2] = 0;
    hf[3] = maxiter + 8;
    for (int i = 4; i < 8; ++i) hf[i] = 0;  // [4]: a bulk-copy wait in a CG kernel gave up
    CK(cudaMemcpyAsync(w.flags.p, hf, sizeof(int) * 8, cudaMemcpyHostToDevice, c->stream));
  }
  {
    const Ctl ctl0 = work_ctl(c, false);
    BlasArgs b = blas_base(c, ctl0);
    b.gate = GATE_NONE;
    b.fin = FIN_INIT;
    if (full) {
      b.be = full->be;
      b.bo = full->bo;
      b.ref_nmass = nmass;
    }
    CK(launch_cg_init(w.VP, w.RP, w.NS, w.nbx_bl * w.G, c->stream, b));
    CK(launch_finalize(ctl0, FIN_INIT, w.nbx_bl, 2, nsys, c->stream));
  }
  return STAG_OK;
}

// run the staged solve eagerly (no graph), polling the device flag
int solve_eager(stag_ctx *c, int maxiter) {
  Work &w = c->w;
  const Ctl ctl = work_ctl(c, false);
  int *hf = (int *)w.h_flags.p;
  const int passes_per_poll = 4;  // the same sequence as the graph body, polled every 4 passes
  const int unroll = solve_unroll();
  for (long long it = 0; it <= (long long)maxiter + 2 * unroll * passes_per_poll; it += unroll * passes_per_poll) {
    for (int i = 0; i < passes_per_poll; ++i) {
      CKS(enqueue_pass(c, c->stream, ctl, unroll));
      CKS(enqueue_update(c, c->stream, ctl));
    }
    CK(cudaMemcpyAsync(hf, w.flags.p, sizeof(int) * 2, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hf[0] == 0) break;
  }
  return STAG_OK;
}

int solve_status(stag_ctx *c, int iters[], double true_res[]);

// copy the solutions and statistics out; the solve's status
int solve_finish(stag_ctx *c, double *const x[], int iters[], double true_res[]) {
  Work &w = c->w;
  const int nsys = w.nsys;
  CK(cudaMemcpyAsync(w.h_st.p, w.st.p, sizeof(SysState) * nsys, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(w.h_flags.p, w.flags.p, sizeof(int) * 8, cudaMemcpyDeviceToHost, c->stream));
  for (int j = 0; j < nsys; ++j) CKS(vec_out(c, w.x64, j, x[j]));
  return solve_status(c, iters, true_res);
}

// after the states and flags were queued for the host: wait, release the L2
// set-aside, and the solve's status with per-system iterations and residuals
int solve_status(stag_ctx *c, int iters[], double true_res[]) {
  Work &w = c->w;
  const int nsys = w.nsys;
  SysState *hs = (SysState *)w.h_st.p;
  int *hf = (int *)w.h_flags.p;
  CK(cudaStreamSynchronize(c->stream));
  c->last_nsys = nsys;
  // the solve's persisting L2 lines back to normal (the next user of L2, or a
  // flush between timed solves, may evict them) and the set-aside released
  if (w.l2p) {
    cudaCtxResetPersistingL2Cache();
    l2_setaside(c, false);
  }
  cudaGetLastError();
  if (hf[4] != 0) {
    c->err = "a CG kernel gave up waiting for its bulk-copied links; the solution is void";
    return STAG_ERR_TIMEOUT;
  }
  int status = STAG_OK;
  for (int j = 0; j < nsys; ++j) {
    if (iters) iters[j] = hs[j].iter;
    if (true_res) true_res[j] = hs[j].true_res;
    if (hs[j].done == -5) status = STAG_ERR_BREAKDOWN;
    else if (hs[j].done != 1 && status == STAG_OK) status = STAG_NOT_CONVERGED;
  }
  if (status == STAG_ERR_BREAKDOWN) c->err = "CG breakdown: <p, A p> not positive or a non-finite residual";
  else if (status == STAG_NOT_CONVERGED) c->err = "iteration cap reached before the tolerance";
  return status;
}

int solve_run(stag_ctx *c, int maxiter);

int solve_impl(stag_ctx *c, const double *const src[], int nrhs, const double masses[], int nmass,
               double tol, int maxiter, int prec, double *const x[], int iters[], double true_res[]) {
  CKS(solve_stage(c, src, nrhs, masses, nmass, tol, maxiter, prec));
  CKS(solve_run(c, maxiter));
  return solve_finish(c, x, iters, true_res);
}

// run the staged solve: one graph launch, or eager launches without graphs
int solve_run(stag_ctx *c, int maxiter) {
  Work &w = c->w;
  bool ran = false;
  if (c->use_graph) {
    if (!w.graph_tried) {
      const int st = build_graph(c);
      if (st != STAG_OK) {
        // conditional nodes unavailable: fall back to eager launches
        w.drop_graph();
        w.graph_tried = true;
        c->use_graph = false;
      }
    }
    if (w.exec) {
      if (w.l2p) l2_setaside(c, true);
      CK(cudaGraphLaunch(w.exec, c->stream));
      ran = true;
    }
  }
  if (!ran) {
    if (w.l2p) l2_setaside(c, true);
    CKS(solve_eager(c, maxiter));
  }
  return STAG_OK;
}

// One FP64 half operator with the mass epilogue on system slots of FP64
// vectors: out[ko] = scale (m4 center[kc] - D in[ki]) on the sites of parity
// par_out (scale = 0: no scaling).  The vectors are views of one system each.
VecArg vec_slot(const VecBuf &v, int k) {
  VecArg a = v.arg();
  a.v = (char *)a.v + cplx_bytes(v.prec) * (size_t)a.sstr * k;
  return a;
}

int apply_m64(stag_ctx *c, int par_out, double m4, double scale, VecArg in, VecArg center, VecArg out) {
  int lanes = 1;
  CKS(tune_lanes(c, P64, 0, P64, 1, 1, 1, c->links64.p, in, out, &lanes));
  DsArgs a = ds_base(c);
  a.links = c->links64.p;
  a.nsys = 1;
  a.ngroups = 1;
  a.ctl = no_ctl();
  a.gate = GATE_NONE;
  a.fin = FIN_NONE;
  a.m4_single = m4;
  a.out_scale = scale;
  a.par_out = par_out;
  a.in = in;
  a.center = center;
  a.out = out;
  CK(launch_dslash(P64, 0, P64, P64, 1, EPI_MDAGM, lanes, ds_blocks(c->Ve, lanes), c->stream, a));
  return STAG_OK;
}

// The full-lattice equation M x = b, M = 2m + D, through the even-site CG:
//   b_s = 2m b_e - D_eo b_o;  (4m^2 - D_eo D_oe) x_e = b_s;  x_o = (b_o - D_oe x_e) / (2m)
// (all FP64 except the CG's inner iteration).  The CG's reference norm is
// 2m |b|: with x_o as above the odd rows of b - M x vanish (to rounding) and
// the even rows are (b_s - A x_e) / (2m), so |b - M x| / |b| = |r_s| / (2m |b|).
int solve_full_impl(stag_ctx *c, const double *const src[], int nrhs, const double masses[], int nmass,
                    double tol, int maxiter, int prec, double *const x[], int iters[], double true_res[]) {
  const int nsys = nrhs * nmass;
  CKS(work_prepare(c, nsys, prec));
  Work &w = c->w;
  const void *lo = nullptr;
  CKS(links_for(c, w.prec, &lo));
  const int Ve = c->Ve;
  const size_t full_bytes = sizeof(double) * 6ull * (size_t)c->V;
  CK(c->full_e.ensure(P64, nrhs, Ve));
  CK(c->full_o.ensure(P64, nrhs, Ve));
  CK(c->full_x.ensure(P64, 1, Ve));
  // full sources -> their even and odd halves
  for (int r = 0; r < nrhs; ++r) {
    const double2 *d = nullptr;
    if (is_device_ptr(src[r])) {
      d = reinterpret_cast<const double2 *>(src[r]);
    } else {
      CK(c->stage_in.ensure(full_bytes));
      CK(cudaMemcpyAsync(c->stage_in.p, src[r], full_bytes, cudaMemcpyHostToDevice, c->stream));
      d = reinterpret_cast<const double2 *>(c->stage_in.p);
    }
    CK(launch_split_full(d, c->full_e.arg(), c->full_o.arg(), r, c->g, c->stream));
  }
  // even-site sources b_s = 2m b_e - D_eo b_o of every system
  for (int r = 0; r < nrhs; ++r)
    for (int k = 0; k < nmass; ++k)
      CKS(apply_m64(c, 0, 2.0 * masses[k], 0.0, vec_slot(c->full_o, r), vec_slot(c->full_e, r),
                    vec_slot(w.b64, r * nmass + k)));
  FullRef ref;
  ref.be = c->full_e.arg();
  ref.bo = c->full_o.arg();
  CKS(solve_start(c, masses, nmass, tol, maxiter, &ref));
  CKS(solve_run(c, maxiter));
  CK(cudaMemcpyAsync(w.h_st.p, w.st.p, sizeof(SysState) * nsys, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(w.h_flags.p, w.flags.p, sizeof(int) * 8, cudaMemcpyDeviceToHost, c->stream));
  // x_o = (b_o - D_oe x_e) / (2m), then both halves into the caller's full vector
  for (int j = 0; j < nsys; ++j) {
    const int r = j / nmass, k = j % nmass;
    CKS(apply_m64(c, 1, 1.0, 1.0 / (2.0 * masses[k]), vec_slot(w.x64, j), vec_slot(c->full_o, r),
                  c->full_x.arg()));
    if (is_device_ptr(x[j])) {
      CK(launch_merge_full(w.x64.arg(), j, c->full_x.arg(), 0, reinterpret_cast<double2 *>(x[j]), c->g,
                           c->stream));
    } else {
      CK(c->stage_out.ensure(full_bytes));
      CK(launch_merge_full(w.x64.arg(), j, c->full_x.arg(), 0, reinterpret_cast<double2 *>(c->stage_out.p), c->g,
                           c->stream));
      CK(cudaMemcpyAsync(x[j], c->stage_out.p, full_bytes, cudaMemcpyDeviceToHost, c->stream));
    }
  }
  return solve_status(c, iters, true_res);
}

// operator calls of the ABI: the FP64 input is rounded to `prec` (per-site
// scaled for FP16/BF16) and the result returned unrounded (FP32 arithmetic),
// or, with STAG_ROUND_OUTPUT set, rounded to `prec` as inside the solver.
int op_impl(stag_ctx *c, int which, int precision, double mass, const double *in, double *out) {
  const bool round_out = (precision & STAG_ROUND_OUTPUT) != 0;
  const int P = precision & 0xff;
  if (!valid_prec(P)) return arg_err(c, "precision must be STAG_FP64/FP32/FP16/BF16");
  if (!in || !out) return arg_err(c, "NULL vector");
  const void *links = nullptr;
  CKS(links_for(c, P, &links));
  const int recon = link_recon(c, P);
  const int VP = (P == P64 || P == P32 || round_out) ? P : P32;
  const int Ve = c->Ve;
  const double2 *d = nullptr;
  CKS(vec_in(c, in, c->stage_in, 0, &d));
  CK(c->api_a.ensure(VP, 1, Ve));
  CK(c->api_b.ensure(VP, 1, Ve));
  CK(c->api_c.ensure(VP, 1, Ve));
  if (VP == P) {
    CK(launch_pack_vec(P, d, c->api_a.arg(), 0, Ve, c->stream));
  } else {
    // round through the storage format, hold the values in FP32
    CK(c->api_c.ensure(P, 1, Ve));
    CK(launch_pack_vec(P, d, c->api_c.arg(), 0, Ve, c->stream));
    CK(launch_convert_vec(P, P32, c->api_c.arg(), c->api_a.arg(), 1, Ve, c->stream));
  }
  DsArgs a = ds_base(c);
  a.links = links;
  a.nsys = 1;
  a.ngroups = 1;
  a.ctl = no_ctl();
  a.gate = GATE_NONE;
  a.fin = FIN_NONE;
  a.m4_single = 4.0 * mass * mass;
  int lanes = 1;
  CKS(tune_lanes(c, P, recon, VP, 1, 1, 1, links, c->api_a.arg(), c->api_b.arg(), &lanes));
  const int nb = ds_blocks(Ve, lanes);
  if (which == 0 || which == 1) {  // 0: D_oe (out odd), 1: D_eo (out even)
    a.par_out = which == 0 ? 1 : 0;
    a.in = c->api_a.arg();
    a.out = c->api_b.arg();
    CK(launch_dslash(P, recon, VP, VP, 1, EPI_PLAIN, lanes, nb, c->stream, a));
  } else {  // M^dag M
    a.par_out = 1;
    a.in = c->api_a.arg();
    a.out = c->api_c.arg();
    CK(c->api_c.ensure(VP, 1, Ve));
    CK(launch_dslash(P, recon, VP, VP, 1, EPI_PLAIN, lanes, nb, c->stream, a));
    a.par_out = 0;
    a.in = c->api_c.arg();
    a.center = c->api_a.arg();
    a.out = c->api_b.arg();
    CK(launch_dslash(P, recon, VP, VP, 1, EPI_MDAGM, lanes, nb, c->stream, a));
  }
  CKS(vec_out(c, c->api_b, 0, out));
  CK(cudaStreamSynchronize(c->stream));
  return STAG_OK;
}

// Multi-shift CG (several masses of each source on one Krylov space), then a
// per-mass mixed-precision refinement:
//  phase 1: the base systems (the smallest mass) run the CG of stag_cg_solve
//    with its reliable updates; the other masses ride on it as shifts (the
//    shift kernel between the two CG kernels) until their estimated residual
//    zeta |r| falls below MS_SHIFT_TOL |b| -- the FP32 recurrences leave them
//    at about eps_32 kappa_s of their own systems, whatever the base does;
//  phase 2: every shifted system is solved from its phase-1 solution as the
//    initial guess (one batched solve; its first step recomputes r = b - A x0
//    in FP64) to the tolerance.
int ms_impl(stag_ctx *c, const double *const src[], int nrhs, const double masses[], int nmass, double tol,
            int maxiter, int prec, double *const x[], int iters[], double true_res[]) {
  int k0 = 0;
  for (int k = 1; k < nmass; ++k)
    if (masses[k] * masses[k] < masses[k0] * masses[k0]) k0 = k;
  std::vector<int> sk;  // user index of each shift
  std::vector<double> sm;
  for (int k = 0; k < nmass; ++k)
    if (k != k0) {
      sk.push_back(k);
      sm.push_back(masses[k]);
    }
  const int nsh = nmass - 1, nsys2 = nrhs * nsh, Ve = c->Ve;
  // phase 1
  CKS(work_prepare(c, nrhs, prec, nsh));
  Work &w = c->w;
  const void *lo = nullptr;
  CKS(links_for(c, w.prec, &lo));
  for (int r = 0; r < nrhs; ++r) {
    const double2 *d = nullptr;
    CKS(vec_in(c, src[r], c->stage_in, 0, &d));
    CK(launch_pack_vec(P64, d, w.b64.arg(), r, Ve, c->stream));
  }
  CK(c->ms_p.ensure(P32, nsys2, Ve));
  CK(c->ms_x.ensure(P32, nsys2, Ve));
  CK(c->ms_sh.ensure(sizeof(ShiftState) * nsys2));
  CK(c->ms_h.ensure(sizeof(ShiftState) * nsys2));
  CK(cudaMemsetAsync(c->ms_p.data.p, 0, cplx_bytes(P32) * 3ull * nsys2 * Ve, c->stream));
  CK(cudaMemsetAsync(c->ms_x.data.p, 0, cplx_bytes(P32) * 3ull * nsys2 * Ve, c->stream));
  ShiftState *hs = (ShiftState *)c->ms_h.p;
  CK(cudaStreamSynchronize(c->stream));  // the pinned staging buffer is free
  for (int r = 0; r < nrhs; ++r)
    for (int q = 0; q < nsh; ++q) {
      ShiftState &h = hs[r * nsh + q];
      memset(&h, 0, sizeof h);
      h.dm4 = 4.0 * sm[q] * sm[q] - 4.0 * masses[k0] * masses[k0];
      h.zeta = h.zeta_prev = h.alpha_prev = 1.0;
      h.active = 1;
    }
  CK(cudaMemcpyAsync(c->ms_sh.p, hs, sizeof(ShiftState) * nsys2, cudaMemcpyHostToDevice, c->stream));
  const double m0[1] = {masses[k0]};
  CKS(solve_start(c, m0, 1, tol, maxiter, nullptr));
  CKS(solve_run(c, maxiter));
  CK(cudaMemcpyAsync(w.h_st.p, w.st.p, sizeof(SysState) * nrhs, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(w.h_flags.p, w.flags.p, sizeof(int) * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(hs, c->ms_sh.p, sizeof(ShiftState) * nsys2, cudaMemcpyDeviceToHost, c->stream));
  for (int r = 0; r < nrhs; ++r) CKS(vec_out(c, w.x64, r, x[r * nmass + k0]));
  std::vector<int> it1(nrhs), it2(nsys2);
  std::vector<double> tr1(nrhs), tr2(nsys2);
  const int st1 = solve_status(c, it1.data(), tr1.data());
  if (st1 < 0) return st1;
  std::vector<int> ms_it(nsys2);
  for (int j = 0; j < nsys2; ++j) ms_it[j] = hs[j].iter;
  // phase 2: the shifted systems from their phase-1 solutions
  CKS(solve_stage(c, src, nrhs, sm.data(), nsh, tol, maxiter, prec));
  CK(launch_convert_vec(P32, P64, c->ms_x.arg(), w.x64.arg(), nsys2, Ve, c->stream));
  CK(launch_mark_update(w.st.p ? (SysState *)w.st.p : nullptr, nsys2, c->stream));
  CKS(enqueue_update(c, c->stream, work_ctl(c, false)));
  CKS(solve_run(c, maxiter));
  CK(cudaMemcpyAsync(w.h_st.p, w.st.p, sizeof(SysState) * nsys2, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(w.h_flags.p, w.flags.p, sizeof(int) * 8, cudaMemcpyDeviceToHost, c->stream));
  for (int r = 0; r < nrhs; ++r)
    for (int q = 0; q < nsh; ++q) CKS(vec_out(c, w.x64, r * nsh + q, x[r * nmass + sk[q]]));
  const int st2 = solve_status(c, it2.data(), tr2.data());
  for (int r = 0; r < nrhs; ++r) {
    if (iters) iters[r * nmass + k0] = it1[r];
    if (true_res) true_res[r * nmass + k0] = tr1[r];
    for (int q = 0; q < nsh; ++q) {
      if (iters) iters[r * nmass + sk[q]] = ms_it[r * nsh + q] + it2[r * nsh + q];
      if (true_res) true_res[r * nmass + sk[q]] = tr2[r * nsh + q];
    }
  }
  if (st2 < 0) return st2;
  return (st1 == STAG_OK && st2 == STAG_OK) ? STAG_OK : STAG_NOT_CONVERGED;
}

// out = D in (FP64) on the sites of parity par_out, one system
int apply_m64_plain(stag_ctx *c, int par_out, VecArg in, VecArg out) {
  int lanes = 1;
  CKS(tune_lanes(c, P64, 0, P64, 1, 1, 1, c->links64.p, in, out, &lanes));
  DsArgs a = ds_base(c);
  a.links = c->links64.p;
  a.nsys = 1;
  a.ngroups = 1;
  a.ctl = no_ctl();
  a.gate = GATE_NONE;
  a.fin = FIN_NONE;
  a.par_out = par_out;
  a.in = in;
  a.out = out;
  CK(launch_dslash(P64, 0, P64, P64, 1, EPI_PLAIN, lanes, ds_blocks(c->Ve, lanes), c->stream, a));
  return STAG_OK;
}

// The fermion force at x_even, every output multiplied by `scale` (the
// chain-rule factor of a caller): grad_links = scale K^dag, lie_force =
// scale f_a, grad_phi = 2 scale x (each may be null; host or device).
int force_impl(stag_ctx *c, const double *x_even, double scale, double *grad_links, double *lie_force,
               double *grad_phi) {
  if (!c->have_links) {
    c->err = "no gauge field: call stag_links_upload first";
    return STAG_ERR_STATE;
  }
  const int Ve = c->Ve;
  const double2 *d = nullptr;
  CKS(vec_in(c, x_even, c->stage_in, 0, &d));
  if (grad_phi) {
    const size_t vb = sizeof(double) * 6ull * Ve;
    if (is_device_ptr(grad_phi)) {
      CK(launch_scale_reals((const double *)d, 2.0 * scale, grad_phi, 6ll * Ve, c->stream));
    } else {
      CK(c->stage_out.ensure(vb));
      CK(launch_scale_reals((const double *)d, 2.0 * scale, (double *)c->stage_out.p, 6ll * Ve, c->stream));
      CK(cudaMemcpyAsync(grad_phi, c->stage_out.p, vb, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));  // stage_out is reused below
    }
  }
  if (!grad_links && !lie_force) {
    CK(cudaStreamSynchronize(c->stream));
    return STAG_OK;
  }
  CK(c->api_a.ensure(P64, 1, Ve));
  CK(c->api_b.ensure(P64, 1, Ve));
  CK(launch_pack_vec(P64, d, c->api_a.arg(), 0, Ve, c->stream));
  // Y = D_oe X (FP64)
  CKS(apply_m64_plain(c, 1, c->api_a.arg(), c->api_b.arg()));
  const size_t gbytes = sizeof(double) * 18ull * 4ull * c->V, lbytes = sizeof(double) * 8ull * 4ull * c->V;
  double2 *gdev = nullptr;
  double *ldev = nullptr;
  const bool g_host = grad_links && !is_device_ptr(grad_links);
  const bool l_host = lie_force && !is_device_ptr(lie_force);
  size_t off = 0;
  if (g_host) off += gbytes;
  if (l_host) off += lbytes;
  if (off) CK(c->stage_out.ensure(off));
  off = 0;
  if (grad_links) {
    gdev = g_host ? (double2 *)c->stage_out.p : (double2 *)grad_links;
    if (g_host) off += gbytes;
  }
  if (lie_force) ldev = l_host ? (double *)((char *)c->stage_out.p + off) : lie_force;
  CK(launch_force(c->g, (const double2 *)c->api_a.data.p, (const double2 *)c->api_b.data.p, c->links64.p, gdev, ldev,
                  scale, c->stream));
  if (g_host) CK(cudaMemcpyAsync(grad_links, gdev, gbytes, cudaMemcpyDeviceToHost, c->stream));
  if (l_host) CK(cudaMemcpyAsync(lie_force, ldev, lbytes, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return STAG_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// ragged batch: several contexts (lattices of different sizes) in one graph
// ---------------------------------------------------------------------------
struct RaggedGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
std::map<std::vector<unsigned long long>, RaggedGraph> g_ragged;
std::mutex g_ragged_mu;
unsigned long long g_next_ctx_id = 1;

void ragged_forget(unsigned long long id) {
  std::lock_guard<std::mutex> lk(g_ragged_mu);
  for (auto it = g_ragged.begin(); it != g_ragged.end();) {
    bool has = false;
    for (size_t k = 0; k < it->first.size(); k += 2) has |= it->first[k] == id;
    if (has) {
      if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
      if (it->second.graph) cudaGraphDestroy(it->second.graph);
      it = g_ragged.erase(it);
    } else {
      ++it;
    }
  }
}

int ragged_impl(const stag_solve_desc *d, int n, double tol, int maxiter, int prec) {
  stag_ctx *c0 = d[0].ctx;
  std::vector<cudaStream_t> saved(n);
  for (int i = 0; i < n; ++i) {
    saved[i] = d[i].ctx->stream;
    d[i].ctx->stream = c0->stream;  // one stream orders the whole batch
  }
  struct Restore {
    const stag_solve_desc *d;
    int n;
    std::vector<cudaStream_t> &s;
    ~Restore() {
      for (int i = 0; i < n; ++i) d[i].ctx->stream = s[i];
    }
  } restore{d, n, saved};
  for (int i = 0; i < n; ++i) {
    stag_ctx *c = d[i].ctx;
    CKS(solve_stage(c, d[i].src, d[i].nrhs, d[i].masses, d[i].nmass, tol, maxiter, prec));
  }
  bool graph_ok = true;
  for (int i = 0; i < n; ++i) graph_ok &= d[i].ctx->use_graph;
  bool ran = false;
  if (graph_ok) {
    std::vector<unsigned long long> key;
    for (int i = 0; i < n; ++i) {
      key.push_back(d[i].ctx->id);
      key.push_back(d[i].ctx->w.gen);
    }
    cudaGraphExec_t exec = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_ragged_mu);
      auto it = g_ragged.find(key);
      if (it != g_ragged.end()) exec = it->second.exec;
    }
    if (!exec) {
      RaggedGraph rg;
      stag_ctx *c = c0;
      CK(cudaGraphCreate(&rg.graph, 0));
      int st = STAG_OK;
      for (int i = 0; i < n && st == STAG_OK; ++i) {
        st = add_solve_loop(d[i].ctx, rg.graph, nullptr, 0, nullptr);
        if (st != STAG_OK) {
          cudaStreamCaptureStatus cs;
          cudaGraph_t tmp = nullptr;
          stag_ctx *ci = d[i].ctx;
          if (ci->cap2 && cudaStreamIsCapturing(ci->cap2, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            cudaStreamEndCapture(ci->cap2, &tmp);
          if (ci->cap && cudaStreamIsCapturing(ci->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            cudaStreamEndCapture(ci->cap, &tmp);
          cudaGetLastError();
        }
      }
      if (st == STAG_OK && cudaGraphInstantiate(&rg.exec, rg.graph, 0) == cudaSuccess) {
        exec = rg.exec;
        std::lock_guard<std::mutex> lk(g_ragged_mu);
        g_ragged[key] = rg;
      } else {
        cudaGetLastError();
        if (rg.graph) cudaGraphDestroy(rg.graph);
      }
    }
    if (exec) {
      stag_ctx *c = c0;
      for (int i = 0; i < n; ++i)
        if (d[i].ctx->w.l2p) l2_setaside(d[i].ctx, true);
      CK(cudaGraphLaunch(exec, c0->stream));
      ran = true;
    }
  }
  if (!ran)
    for (int i = 0; i < n; ++i) {
      if (d[i].ctx->w.l2p) l2_setaside(d[i].ctx, true);
      CKS(solve_eager(d[i].ctx, maxiter));
    }
  int status = STAG_OK;
  for (int i = 0; i < n; ++i) {
    const int st = solve_finish(d[i].ctx, d[i].x, d[i].iters, d[i].true_res);
    if (st < 0 || (st == STAG_NOT_CONVERGED && status == STAG_OK)) status = st;
  }
  if (status != STAG_OK) {
    for (int i = 0; i < n; ++i)
      if (!d[i].ctx->err.empty()) {
        c0->err = d[i].ctx->err;
        break;
      }
  }
  return status;
}

// Internal accessors used by noalloc.cu (not part of the C ABI).
namespace stag {
int ctx_fp64_links(const stag_ctx *c, const void **links, cudaStream_t *stream) {
  if (!c->have_links) return STAG_ERR_STATE;
  *links = c->links64.p;
  *stream = c->stream;
  return STAG_OK;
}
void ctx_set_error(stag_ctx *c, const char *msg) { c->err = msg; }
Geom ctx_geom(const stag_ctx *c) { return c->g; }
int ctx_device(const stag_ctx *c) { return c->device; }
}  // namespace stag

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int stag_abi_version(void) { return STAG_ABI_VERSION; }

const char *stag_status_string(int s) {
  switch (s) {
    case STAG_OK: return "STAG_OK";
    case STAG_NOT_CONVERGED: return "STAG_NOT_CONVERGED";
    case STAG_ERR_ARG: return "STAG_ERR_ARG";
    case STAG_ERR_CUDA: return "STAG_ERR_CUDA";
    case STAG_ERR_OOM: return "STAG_ERR_OOM";
    case STAG_ERR_NOT_SU3: return "STAG_ERR_NOT_SU3";
    case STAG_ERR_BREAKDOWN: return "STAG_ERR_BREAKDOWN";
    case STAG_ERR_TIMEOUT: return "STAG_ERR_TIMEOUT";
    case STAG_ERR_STATE: return "STAG_ERR_STATE";
  }
  return "STAG_UNKNOWN_STATUS";
}

const char *stag_last_error(const stag_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

int stag_create(const int dims[4], int flags, void *cuda_stream, stag_ctx **out) {
  if (!out || !dims) return STAG_ERR_ARG;
  *out = nullptr;
  long long V = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 2 || (dims[m] & 1)) return STAG_ERR_ARG;
    V *= dims[m];
  }
  if (V / 2 >= (1ll << 31) / 3) return STAG_ERR_ARG;
  if (flags & ~(STAG_ANTIPERIODIC_T | STAG_RECON12)) return STAG_ERR_ARG;
  stag_ctx *c = new stag_ctx();
  for (int m = 0; m < 4; ++m) c->dims[m] = dims[m];
  c->flags = flags;
  c->stream = (cudaStream_t)cuda_stream;
  c->V = V;
  c->Ve = (int)(V / 2);
  c->g.L0 = dims[0];
  c->g.L1 = dims[1];
  c->g.L2 = dims[2];
  c->g.L3 = dims[3];
  c->g.Lxh = dims[0] / 2;
  c->g.Ve = c->Ve;
  c->g.ap = (flags & STAG_ANTIPERIODIC_T) ? 1 : 0;
  c->g.dLxh = make_fastdiv((unsigned)(dims[0] / 2));
  c->g.dL1 = make_fastdiv((unsigned)dims[1]);
  c->g.dL2 = make_fastdiv((unsigned)dims[2]);
  {
    std::lock_guard<std::mutex> lk(g_ragged_mu);
    c->id = g_next_ctx_id++;
  }
  const char *eager = getenv("STAG_EAGER");
  c->use_graph = !(eager && eager[0] == '1');
  const char *pdl = getenv("STAG_PDL");
  c->pdl = !(pdl && pdl[0] == '0');
  const char *fold = getenv("STAG_FOLD");
  c->fold = !(fold && fold[0] == '0');
  const char *persist = getenv("STAG_PERSIST");
  c->persist = !(persist && persist[0] == '0');
  const char *tma = getenv("STAG_TMA");
  // STAG_TMA = 0, 1 or 2 fixes the link path of the single-system CG kernels,
  // t lets the tuner try all three; by default it tries 0 and 2 (the bulk
  // copies through shared memory, 1, measured slower at FP32 and FP16: shared
  // memory caps the sites in flight per SM below what the registers hold)
  if (tma && (tma[0] == '0' || tma[0] == '1' || tma[0] == '2') && tma[1] == 0) c->tma_modes = 1 << (tma[0] - '0');
  else if (tma && tma[0] == 't' && tma[1] == 0) c->tma_modes = 0b111;
  const char *giveup = getenv("STAG_TEST_WAIT_GIVEUP");
  c->wait_giveup = (giveup && giveup[0] == '1') ? 1 : 0;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return STAG_ERR_CUDA;
  }
  {
    // STAG_L2PERSIST = 0 off, 1 the links persist, 2 the Krylov vectors persist
    const char *l2p = getenv("STAG_L2PERSIST");
    c->l2persist = !(l2p && l2p[0] == '0');
    if (l2p && l2p[0] == '1') c->l2_modes = 0b010;
    if (l2p && l2p[0] == '2') c->l2_modes = 0b100;
    int maxp = 0, maxw = 0;
    if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, c->device) != cudaSuccess)
      maxp = maxw = 0;
    cudaGetLastError();
    if (c->l2persist && maxp > 0 && maxw > 0) {
      c->l2_max_persist = (size_t)maxp;
      c->l2_max_window = (size_t)maxw;
    }
    if (c->l2_max_persist == 0) c->l2persist = false;
  }
  *out = c;
  return STAG_OK;
}

int stag_destroy(stag_ctx *c) {
  if (!c) return STAG_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  ragged_forget(c->id);
  c->w.drop_graph();
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->cap2) cudaStreamDestroy(c->cap2);
  delete c;
  return STAG_OK;
}

int stag_links_upload(stag_ctx *c, const double *links) {
  if (!c) return STAG_ERR_ARG;
  if (!links) return arg_err(c, "NULL links");
  CK(cudaSetDevice(c->device));
  const size_t bytes = sizeof(double) * 18ull * 4ull * c->V;
  CK(c->links_canon.ensure(bytes));
  CK(cudaMemcpyAsync(c->links_canon.p, links, bytes, cudaMemcpyDefault, c->stream));
  if (c->flags & STAG_RECON12) {
    CK(c->defect.ensure(sizeof(unsigned long long)));
    CK(cudaMemsetAsync(c->defect.p, 0, sizeof(unsigned long long), c->stream));
    CK(launch_su3_defect(reinterpret_cast<const double2 *>(c->links_canon.p), 4ll * c->V,
                         (unsigned long long *)c->defect.p, c->stream));
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, c->defect.p, sizeof bits, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double d;
    memcpy(&d, &bits, sizeof d);
    if (!(d <= 1e-12)) {
      char buf[160];
      snprintf(buf, sizeof buf, "links are not SU(3) (defect %.3e > 1e-12); reconstruct-12 needs SU(3)", d);
      c->err = buf;
      c->have_links = false;
      return STAG_ERR_NOT_SU3;
    }
  }
  CK(c->links64.ensure(cplx_bytes(P64) * 9ull * 8ull * c->Ve));
  CK(launch_pack_links(P64, 0, reinterpret_cast<const double2 *>(c->links_canon.p), c->links64.p, c->g,
                       c->stream));
  for (int p = 0; p < 4; ++p) c->lo_ok[p][0] = c->lo_ok[p][1] = c->tile_ok[p][0] = c->tile_ok[p][1] = false;
  c->have_links = true;
  c->w.drop_graph();  // the graph holds link pointers of the reduced-precision copies
  CK(cudaStreamSynchronize(c->stream));
  return STAG_OK;
}

int stag_dslash_oe(stag_ctx *c, int precision, const double *in_even, double *out_odd) {
  if (!c) return STAG_ERR_ARG;
  CK(cudaSetDevice(c->device));
  return op_impl(c, 0, precision, 0.0, in_even, out_odd);
}

int stag_dslash_eo(stag_ctx *c, int precision, const double *in_odd, double *out_even) {
  if (!c) return STAG_ERR_ARG;
  CK(cudaSetDevice(c->device));
  return op_impl(c, 1, precision, 0.0, in_odd, out_even);
}

int stag_mdagm(stag_ctx *c, int precision, double mass, const double *in_even, double *out_even) {
  if (!c) return STAG_ERR_ARG;
  CK(cudaSetDevice(c->device));
  return op_impl(c, 2, precision, mass, in_even, out_even);
}

int stag_cg_solve(stag_ctx *c, const double *const src[], int nrhs, const double masses[], int nmass,
                  double tol, int maxiter, int precision, double *const x[], int iters[],
                  double true_res[]) {
  if (!c) return STAG_ERR_ARG;
  if (!src || !masses || !x) return arg_err(c, "NULL argument");
  if (nrhs < 1 || nmass < 1) return arg_err(c, "nrhs and nmass must be >= 1");
  if ((long long)nrhs * nmass > 4096) return arg_err(c, "at most 4096 systems per solve");
  if (!(tol > 0.0) || !(tol < 1.0)) return arg_err(c, "tol must be in (0, 1)");
  if (maxiter < 1) return arg_err(c, "maxiter must be >= 1");
  {
    int a_, b_, c_;
    if (!solver_precs(precision, &a_, &b_, &c_))
      return arg_err(c, "precision must be STAG_FP64/FP32/FP16/BF16, reduced precisions optionally | "
                        "STAG_VEC_FP16 / STAG_VEC_BF16 (or FP16/BF16 | STAG_HALF_VECTORS)");
  }
  for (int r = 0; r < nrhs; ++r)
    if (!src[r]) return arg_err(c, "NULL source");
  for (int j = 0; j < nrhs * nmass; ++j)
    if (!x[j]) return arg_err(c, "NULL solution buffer");
  for (int k = 0; k < nmass; ++k)
    if (!std::isfinite(masses[k])) return arg_err(c, "non-finite mass");
  CK(cudaSetDevice(c->device));
  return solve_impl(c, src, nrhs, masses, nmass, tol, maxiter, precision, x, iters, true_res);
}

int stag_npr_contract(stag_ctx *c, const int spin_taste[4], const double *chibar1, const double *chi2,
                      const double *chibar3, const double *chi4, double *O_hyp, double *O_sum) {
  if (!c) return STAG_ERR_ARG;
  if (!spin_taste || !chibar1 || !chi2 || !chibar3 || !chi4 || (!O_hyp && !O_sum))
    return arg_err(c, "NULL argument");
  for (int k = 0; k < 4; ++k)
    if (spin_taste[k] < 0 || spin_taste[k] > 15) return arg_err(c, "spin/taste masks are 4-bit (0..15)");
  CK(cudaSetDevice(c->device));
  if (!c->have_links) {
    c->err = "no gauge field: call stag_links_upload first";
    return STAG_ERR_STATE;
  }
  const size_t fb = sizeof(double) * 6ull * (size_t)c->V;
  const long long nh = c->V / 16;
  const double *f[4] = {chibar1, chi2, chibar3, chi4};
  const double2 *d[4];
  CK(c->npr_f.ensure(4 * fb));
  for (int k = 0; k < 4; ++k) {
    if (is_device_ptr(f[k])) {
      d[k] = reinterpret_cast<const double2 *>(f[k]);
    } else {
      CK(cudaMemcpyAsync((char *)c->npr_f.p + k * fb, f[k], fb, cudaMemcpyHostToDevice, c->stream));
      d[k] = reinterpret_cast<const double2 *>((char *)c->npr_f.p + k * fb);
    }
  }
  CK(c->npr_o.ensure(sizeof(double2) * (size_t)(nh + 1)));
  double2 *out = (O_hyp && is_device_ptr(O_hyp)) ? reinterpret_cast<double2 *>(O_hyp) : (double2 *)c->npr_o.p;
  double2 *sum = (double2 *)c->npr_o.p + nh;
  CK(launch_npr(c->dims, reinterpret_cast<const double2 *>(c->links_canon.p), spin_taste, d[0], d[1], d[2], d[3],
                out, O_sum ? sum : nullptr, c->stream));
  if (O_hyp && out == (double2 *)c->npr_o.p)
    CK(cudaMemcpyAsync(O_hyp, out, sizeof(double2) * (size_t)nh, cudaMemcpyDeviceToHost, c->stream));
  if (O_sum) CK(cudaMemcpyAsync(O_sum, sum, sizeof(double2), cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return STAG_OK;
}

int stag_hyp_smear(stag_ctx *c, const double alpha[3], const double *links_in, double *links_out) {
  if (!c) return STAG_ERR_ARG;
  if (!links_in || !links_out) return arg_err(c, "NULL links");
  double a[3] = {0.75, 0.6, 0.3};
  if (alpha) {
    for (int k = 0; k < 3; ++k) {
      if (!std::isfinite(alpha[k])) return arg_err(c, "non-finite smearing parameter");
      a[k] = alpha[k];
    }
  }
  CK(cudaSetDevice(c->device));
  const size_t bytes = sizeof(double) * 18ull * 4ull * c->V;
  const bool in_dev = is_device_ptr(links_in), out_dev = is_device_ptr(links_out);
  CK(c->hyp_b.ensure(sizeof(double) * 18ull * 12ull * c->V));
  CK(c->hyp_t.ensure(sizeof(double) * 18ull * 12ull * c->V));
  if (!in_dev || !out_dev) CK(c->hyp_io.ensure(bytes));
  const double2 *U = reinterpret_cast<const double2 *>(links_in);
  if (!in_dev) {
    CK(cudaMemcpyAsync(c->hyp_io.p, links_in, bytes, cudaMemcpyHostToDevice, c->stream));
    U = reinterpret_cast<const double2 *>(c->hyp_io.p);
  }
  double2 *out = out_dev ? reinterpret_cast<double2 *>(links_out) : reinterpret_cast<double2 *>(c->hyp_io.p);
  CK(launch_hyp(c->dims, U, a, (double2 *)c->hyp_b.p, (double2 *)c->hyp_t.p, out, c->stream));
  if (!out_dev) CK(cudaMemcpyAsync(links_out, c->hyp_io.p, bytes, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return STAG_OK;
}

int stag_cg_solve_multishift(stag_ctx *c, const double *const src[], int nrhs, const double masses[], int nmass,
                             double tol, int maxiter, int precision, double *const x[], int iters[],
                             double true_res[]) {
  if (!c) return STAG_ERR_ARG;
  if (!src || !masses || !x) return arg_err(c, "NULL argument");
  if (nrhs < 1 || nmass < 1) return arg_err(c, "nrhs and nmass must be >= 1");
  if ((long long)nrhs * nmass > 4096) return arg_err(c, "at most 4096 systems per solve");
  if (!(tol > 0.0) || !(tol < 1.0)) return arg_err(c, "tol must be in (0, 1)");
  if (maxiter < 1) return arg_err(c, "maxiter must be >= 1");
  {
    int lp, vp, rp;
    if (!solver_precs(precision, &lp, &vp, &rp)) return arg_err(c, "bad solver precision");
    if (rp != P32) return arg_err(c, "multi-shift CG needs a reduced-precision inner iteration (not STAG_FP64)");
  }
  for (int r = 0; r < nrhs; ++r)
    if (!src[r]) return arg_err(c, "NULL source");
  for (int j = 0; j < nrhs * nmass; ++j)
    if (!x[j]) return arg_err(c, "NULL solution buffer");
  for (int k = 0; k < nmass; ++k)
    if (!std::isfinite(masses[k])) return arg_err(c, "non-finite mass");
  CK(cudaSetDevice(c->device));
  if (!c->have_links) {
    c->err = "no gauge field: call stag_links_upload first";
    return STAG_ERR_STATE;
  }
  if (nmass == 1) return solve_impl(c, src, nrhs, masses, nmass, tol, maxiter, precision, x, iters, true_res);
  return ms_impl(c, src, nrhs, masses, nmass, tol, maxiter, precision, x, iters, true_res);
}

int stag_solve_full(stag_ctx *c, const double *const src[], int nrhs, const double masses[], int nmass,
                    double tol, int maxiter, int precision, double *const x[], int iters[], double true_res[]) {
  if (!c) return STAG_ERR_ARG;
  if (!src || !masses || !x) return arg_err(c, "NULL argument");
  if (nrhs < 1 || nmass < 1) return arg_err(c, "nrhs and nmass must be >= 1");
  if ((long long)nrhs * nmass > 4096) return arg_err(c, "at most 4096 systems per solve");
  if (!(tol > 0.0) || !(tol < 1.0)) return arg_err(c, "tol must be in (0, 1)");
  if (maxiter < 1) return arg_err(c, "maxiter must be >= 1");
  {
    int a_, b_, c_;
    if (!solver_precs(precision, &a_, &b_, &c_)) return arg_err(c, "bad solver precision");
  }
  for (int r = 0; r < nrhs; ++r)
    if (!src[r]) return arg_err(c, "NULL source");
  for (int j = 0; j < nrhs * nmass; ++j)
    if (!x[j]) return arg_err(c, "NULL solution buffer");
  for (int k = 0; k < nmass; ++k)
    if (!(masses[k] > 0.0) || !std::isfinite(masses[k])) return arg_err(c, "masses must be finite and > 0");
  CK(cudaSetDevice(c->device));
  if (!c->have_links) {
    c->err = "no gauge field: call stag_links_upload first";
    return STAG_ERR_STATE;
  }
  return solve_full_impl(c, src, nrhs, masses, nmass, tol, maxiter, precision, x, iters, true_res);
}

int stag_cg_solve_ragged(const stag_solve_desc *descs, int ndesc, double tol, int maxiter, int precision) {
  if (!descs || ndesc < 1) return STAG_ERR_ARG;
  stag_ctx *c = descs[0].ctx;
  if (!c) return STAG_ERR_ARG;
  if (!(tol > 0.0) || !(tol < 1.0)) return arg_err(c, "tol must be in (0, 1)");
  if (maxiter < 1) return arg_err(c, "maxiter must be >= 1");
  {
    int a_, b_, c_;
    if (!solver_precs(precision, &a_, &b_, &c_)) return arg_err(c, "bad solver precision");
  }
  for (int i = 0; i < ndesc; ++i) {
    const stag_solve_desc &d = descs[i];
    if (!d.ctx || !d.src || !d.masses || !d.x || d.nrhs < 1 || d.nmass < 1) return arg_err(c, "bad ragged entry");
    if ((long long)d.nrhs * d.nmass > 4096) return arg_err(c, "at most 4096 systems per lattice");
    if (d.ctx->device != c->device) return arg_err(c, "all lattices of a ragged batch must be on one device");
    for (int q = 0; q < i; ++q)
      if (descs[q].ctx == d.ctx) return arg_err(c, "a context appears twice in a ragged batch");
    for (int r = 0; r < d.nrhs; ++r)
      if (!d.src[r]) return arg_err(c, "NULL source");
    for (int j = 0; j < d.nrhs * d.nmass; ++j)
      if (!d.x[j]) return arg_err(c, "NULL solution buffer");
    for (int k = 0; k < d.nmass; ++k)
      if (!std::isfinite(d.masses[k])) return arg_err(c, "non-finite mass");
  }
  CK(cudaSetDevice(c->device));
  return ragged_impl(descs, ndesc, tol, maxiter, precision);
}

int stag_force(stag_ctx *c, const double *x_even, double *grad_links, double *lie_force) {
  if (!c) return STAG_ERR_ARG;
  if (!x_even) return arg_err(c, "NULL solution vector");
  if (!grad_links && !lie_force) return arg_err(c, "no output requested");
  CK(cudaSetDevice(c->device));
  return force_impl(c, x_even, 1.0, grad_links, lie_force, nullptr);
}

int stag_action_backward(stag_ctx *c, const double *x_even, double gS, double *grad_links, double *grad_phi) {
  if (!c) return STAG_ERR_ARG;
  if (!x_even) return arg_err(c, "NULL solution vector");
  if (!grad_links && !grad_phi) return arg_err(c, "no output requested");
  if (!std::isfinite(gS)) return arg_err(c, "non-finite gS");
  CK(cudaSetDevice(c->device));
  return force_impl(c, x_even, gS, grad_links, nullptr, grad_phi);
}

int stag_action(stag_ctx *c, double mass, const double *phi_even, const double *x_even, double *S) {
  if (!c) return STAG_ERR_ARG;
  if (!phi_even || !x_even || !S) return arg_err(c, "NULL argument");
  if (!std::isfinite(mass)) return arg_err(c, "non-finite mass");
  CK(cudaSetDevice(c->device));
  if (!c->have_links) {
    c->err = "no gauge field: call stag_links_upload first";
    return STAG_ERR_STATE;
  }
  const int Ve = c->Ve;
  const size_t vb = sizeof(double) * 6ull * Ve;
  const double2 *dphi = nullptr, *dx = nullptr;
  CK(c->stage_in.ensure(2 * vb));  // both host inputs share it: no regrowth between the two
  CKS(vec_in(c, phi_even, c->stage_in, 0, &dphi));
  CKS(vec_in(c, x_even, c->stage_in, vb, &dx));
  CK(c->api_a.ensure(P64, 1, Ve));
  CK(c->api_b.ensure(P64, 1, Ve));
  CK(c->api_c.ensure(P64, 1, Ve));
  CK(c->full_x.ensure(P64, 1, Ve));
  CK(launch_pack_vec(P64, dx, c->api_a.arg(), 0, Ve, c->stream));
  CK(launch_pack_vec(P64, dphi, c->full_x.arg(), 0, Ve, c->stream));
  // t = D_oe x, A x = 4 m^2 x - D_eo t (FP64)
  CKS(apply_m64_plain(c, 1, c->api_a.arg(), c->api_c.arg()));
  CKS(apply_m64(c, 0, 4.0 * mass * mass, 0.0, c->api_c.arg(), c->api_a.arg(), c->api_b.arg()));
  CK(c->red.ensure(sizeof(double) * (2ull * action_blocks(Ve) + 1)));
  double *part = (double *)c->red.p;
  double *dS = part + 2ll * action_blocks(Ve);
  CK(launch_action(c->full_x.arg(), c->api_a.arg(), c->api_b.arg(), Ve, part, dS, c->stream));
  CK(cudaMemcpyAsync(S, dS, sizeof(double), cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return STAG_OK;
}

int stag_solve_stats(const stag_ctx *c, int sys, int *iters, int *reliable_updates, double *true_res) {
  if (!c || c->last_nsys <= 0 || sys < 0 || sys >= c->last_nsys) return STAG_ERR_ARG;
  const SysState *hs = (const SysState *)c->w.h_st.p;
  if (iters) *iters = hs[sys].iter;
  if (reliable_updates) *reliable_updates = hs[sys].n_updates;
  if (true_res) *true_res = hs[sys].true_res;
  return STAG_OK;
}

int stag_solve_form(const stag_ctx *c, int out[8]) {
  if (!c || !out || c->w.nsys <= 0) return STAG_ERR_ARG;
  const Work &w = c->w;
  out[0] = w.NS;
  out[1] = w.G;
  out[2] = w.lanes_k1;
  out[3] = w.lanes_k2;
  out[4] = w.tma;
  out[5] = w.l2p;
  out[6] = solve_unroll();
  out[7] = w.mrhs ? 1 : (w.nrhs_sl == 24 ? 3 : (w.nrhs_sl ? 2 : 0));
  if (w.nrhs_sl) {
    out[0] = w.nsys;  // every system in every block
    out[1] = 1;
  }
  return STAG_OK;
}

int stag_solve_counters(const stag_ctx *c, int *loop_passes, int *update_steps) {
  if (!c || c->last_nsys <= 0) return STAG_ERR_ARG;
  const int *hf = (const int *)c->w.h_flags.p;
  if (loop_passes) *loop_passes = hf[2];
  if (update_steps) *update_steps = hf[5];
  return STAG_OK;
}

int stag_time_cg_kernel(stag_ctx *c, int precision, int kernel, int nlaunch, double *ms_per_launch,
                        double *bytes_per_launch) {
  if (!c) return STAG_ERR_ARG;
  int LP_, VP_, RP_;
  if (!solver_precs(precision, &LP_, &VP_, &RP_) || nlaunch < 1 || !ms_per_launch || (kernel != 0 && kernel != 1))
    return arg_err(c, "bad argument");
  CK(cudaSetDevice(c->device));
  const int nsys = c->w.nsys > 0 && c->w.prec == LP_ && c->w.VP == VP_ ? c->w.nsys : 1;
  CKS(work_prepare(c, nsys, precision));
  Work &w = c->w;
  const void *lo = nullptr;
  CKS(links_for(c, w.prec, &lo));
  // the two kernels with the solver's launch configuration (state zeroed:
  // alpha = beta = 0, every system processed)
  DsArgs a1 = ds_base(c);
  a1.links = lo;
  a1.nsys = w.nsys;
  a1.ngroups = w.G;
  a1.ctl = work_ctl(c, false);
  a1.gate = GATE_NONE;
  a1.fin = FIN_NONE;
  a1.aux = w.r.arg();
  a1.xlo = w.x.arg();
  a1.pdl = c->pdl ? 1 : 0;  // launched as in the solve
  if (w.tma) CKS(links_tile_for(c, w.prec, &w.links_tile));
  a1.tma = w.tma;
  a1.links_tile = w.links_tile;
  a1.ntile = link_tiles(c->Ve);
  set_l2_window(c, w.prec, w.tma, w.l2p, a1);
  DsArgs a2 = a1;
  a1.par_out = 1;
  const int epi1 = (w.VP == w.RP) ? EPI_CG_K1R : EPI_CG_K1;
  a1.in = (w.VP == w.RP) ? w.r.arg() : w.p.arg();
  a1.out = w.t.arg();
  a2.par_out = 0;
  a2.in = w.t.arg();
  a2.center = w.p.arg();
  // As in the solve's folded loop, each kernel first finishes its
  // predecessor's reduction in every block (fold_state over the other
  // kernel's partials, states double-buffered); GATE_NONE keeps every system
  // processed whatever the (zeroed, meaningless) states say, so the timing
  // holds the fold's reads and arithmetic and the whole kernel body.
  const bool folded = c->fold && !w.nrhs_sl;
  SysState *S[2] = {(SysState *)w.st.p, (SysState *)w.st2.p};
  double *PA = (double *)w.partials.p, *PB = (double *)w.partials2.p;
  const bool rec1 = (w.VP == w.RP);
  int cur = 0;
  auto prep = [&](int k) {
    if (!folded) return;
    DsArgs &x = k == 0 ? a1 : a2;
    x.ctl.st = S[cur];
    x.ctl.partials = k == 0 ? PA : PB;
    x.fold = k == 0 ? FIN_NORM : (rec1 ? FIN_ALPHA_R : FIN_ALPHA);
    x.fold_partials = k == 0 ? PB : PA;
    x.fold_nbx = k == 0 ? w.nbx_k2 : w.nbx_k1;
    x.fold_nv = (k == 0 || !rec1) ? 2 : 1;
    x.st_out = S[1 - cur];
    cur = 1 - cur;
  };
  // alternate them as the iteration does (so each starts with the cache the
  // other leaves), an event between every two launches
  std::vector<cudaEvent_t> ev(2 * (size_t)nlaunch + 1, nullptr);
  int st = STAG_OK;
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) st = fail(c, STAG_ERR_CUDA, "cudaEventCreate", cudaGetLastError());
  for (int i = 0; i < 2 && st == STAG_OK; ++i) {  // warm-up pair
    prep(0);
    if (launch_cg(c, 0, epi1, c->stream, a1) != cudaSuccess) st = fail(c, STAG_ERR_CUDA, "launch", cudaGetLastError());
    prep(1);
    if (st == STAG_OK && launch_cg(c, 1, EPI_CG_K2, c->stream, a2) != cudaSuccess)
      st = fail(c, STAG_ERR_CUDA, "launch", cudaGetLastError());
  }
  if (w.l2p) l2_setaside(c, true);
  if (st == STAG_OK && cudaEventRecord(ev[0], c->stream) != cudaSuccess)
    st = fail(c, STAG_ERR_CUDA, "cudaEventRecord", cudaGetLastError());
  for (int i = 0; i < nlaunch && st == STAG_OK; ++i) {
    prep(0);
    if (launch_cg(c, 0, epi1, c->stream, a1) != cudaSuccess ||
        cudaEventRecord(ev[2 * i + 1], c->stream) != cudaSuccess)
      st = fail(c, STAG_ERR_CUDA, "launch", cudaGetLastError());
    prep(1);
    if (st == STAG_OK && (launch_cg(c, 1, EPI_CG_K2, c->stream, a2) != cudaSuccess ||
                          cudaEventRecord(ev[2 * i + 2], c->stream) != cudaSuccess))
      st = fail(c, STAG_ERR_CUDA, "launch", cudaGetLastError());
  }
  double tot = 0.0, tot_other = 0.0;
  if (st == STAG_OK && cudaEventSynchronize(ev.back()) != cudaSuccess)
    st = fail(c, STAG_ERR_CUDA, "cudaEventSynchronize", cudaGetLastError());
  for (int i = 0; i < nlaunch && st == STAG_OK; ++i) {
    float ms = 0.f, mo = 0.f;
    if (cudaEventElapsedTime(&ms, ev[2 * i + kernel], ev[2 * i + kernel + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&mo, ev[2 * i + 1 - kernel], ev[2 * i + 2 - kernel]) != cudaSuccess)
      st = fail(c, STAG_ERR_CUDA, "cudaEventElapsedTime", cudaGetLastError());
    tot += ms;
    tot_other += mo;
  }
  // An event between two launches stops the programmatic dependent launch
  // that, in the solve, overlaps each kernel's launch with its predecessor's
  // tail; so the same pairs run again with events only around the whole
  // sequence, and each kernel is given its share (from the separated
  // timings) of that pair time.
  double pair_ms = 0.0;
  if (st == STAG_OK && c->pdl) {
    if (cudaEventRecord(ev[0], c->stream) != cudaSuccess)
      st = fail(c, STAG_ERR_CUDA, "cudaEventRecord", cudaGetLastError());
    for (int i = 0; i < nlaunch && st == STAG_OK; ++i) {
      prep(0);
      if (launch_cg(c, 0, epi1, c->stream, a1) != cudaSuccess) st = fail(c, STAG_ERR_CUDA, "launch", cudaGetLastError());
      prep(1);
      if (st == STAG_OK && launch_cg(c, 1, EPI_CG_K2, c->stream, a2) != cudaSuccess)
        st = fail(c, STAG_ERR_CUDA, "launch", cudaGetLastError());
    }
    float ms = 0.f;
    if (st == STAG_OK && (cudaEventRecord(ev[1], c->stream) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
                          cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess))
      st = fail(c, STAG_ERR_CUDA, "pair timing", cudaGetLastError());
    pair_ms = ms;
  }
  if (st == STAG_OK && pair_ms > 0.0 && tot + tot_other > 0.0) tot = pair_ms * tot / (tot + tot_other);
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  if (w.l2p) {
    cudaCtxResetPersistingL2Cache();
    l2_setaside(c, false);
  }
  cudaGetLastError();
  if (st != STAG_OK) return st;
  *ms_per_launch = tot / nlaunch;
  if (bytes_per_launch) {
    const double lb = (double)cplx_bytes(w.prec) * (w.recon ? 6 : 9);
    const double vb = (double)cplx_bytes(w.VP) * 3 + ((w.VP == P16 || w.VP == PBF) ? 4 : 0);
    const double rb = (double)cplx_bytes(w.RP) * 3;
    // links once; the gathered vector once (through cache); then
    //   first kernel: t_old read (recurrence) or p_old gathered (gather form), t written
    //   second kernel: p read and written, r and x_lo read and written
    const double per = (kernel == 0) ? (2.0 * vb + rb) : (3.0 * vb + 4.0 * rb);
    // algorithmic: the links once, whatever the grouping of the systems
    *bytes_per_launch = (double)c->Ve * (8.0 * lb + w.nsys * per);
  }
  return STAG_OK;
}

int stag_time_dslash(stag_ctx *c, int precision, int nlaunch, double *ms_per_launch, double *bytes_per_launch) {
  return stag_time_cg_kernel(c, precision, 0, nlaunch, ms_per_launch, bytes_per_launch);
}

}  // extern "C"
