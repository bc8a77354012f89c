// noalloc.cu -- stag_mdagm_dot_noalloc: the even-site normal operator with its
// FP64 inner product, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a memory budget
// owned by another allocator (a framework's caching allocator that already
// holds the device memory), or code that must not allocate between a set-up
// phase and a time-critical loop.  This entry point allocates nothing: the
// caller passes every vector, and the only scratch -- the per-block partial
// sums and the ticket of the deterministic cross-block reduction -- lives in a
// fixed-size file-scope __device__ array that every GPU loading the library
// holds until the process exits.
//
// Limits and rules:
//   * at most NA_MAX_BLOCKS blocks of NA_BT threads, i.e. Ve <= 8 388 608
//     sites per parity (a 64^3 x 64 lattice); larger lattices get STAG_ERR_ARG;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (once per device, that device current); make that
//     first call before any stream capture;
//   * all calls share the one array: the ticket is cleared at the start of
//     every call, and calls whose work overlaps on the GPU (different streams,
//     or several host threads) race on it -- serialise them.
#include <mutex>

#include "launch.h"
#include "stag.h"

namespace stag {
int ctx_fp64_links(const stag_ctx *c, const void **links, cudaStream_t *stream);
void ctx_set_error(stag_ctx *c, const char *msg);
Geom ctx_geom(const stag_ctx *c);
int ctx_device(const stag_ctx *c);
}  // namespace stag

using namespace stag;

namespace {

constexpr int NA_BT = 128;
constexpr int NA_MAX_BLOCKS = 65536;
constexpr size_t NA_TICKET_BYTES = 256;  // the ticket, padded to keep the partials 256-byte aligned
constexpr size_t NA_SCRATCH_BYTES = NA_TICKET_BYTES + sizeof(double) * NA_MAX_BLOCKS;  // 512.25 KiB

static __device__ __align__(256) unsigned char g_na_scratch[NA_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
unsigned char *g_na_ptr[NA_MAX_DEVICES] = {nullptr};

// device address of g_na_scratch on `device` (which must be current); looked up once per device
cudaError_t na_scratch(int device, unsigned char **out) {
  if (device < 0 || device >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_na_mutex);
  if (!g_na_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[device] = (unsigned char *)p;
  }
  *out = g_na_ptr[device];
  return cudaSuccess;
}

__device__ __forceinline__ void na_load(const double2 *v, int s, double (&x)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double2 w = v[(long long)s * 3 + c];
    x[2 * c] = w.x;
    x[2 * c + 1] = w.y;
  }
}

__device__ __forceinline__ void na_store(double2 *v, int s, const double (&x)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) v[(long long)s * 3 + c] = make_double2(x[2 * c], x[2 * c + 1]);
}

// D applied at output site s of parity P to the ABI-layout vector `in` (FP64)
__device__ __forceinline__ void na_hop_sum(const Geom &g, const void *links, int P, int s, const double2 *in,
                                           double (&acc)[6]) {
  int x[4];
  site_coords(g, P, s, x);
  const int Ls[4] = {g.L0, g.L1, g.L2, g.L3};
#pragma unroll
  for (int i = 0; i < 6; ++i) acc[i] = 0.0;
  int eta_bits = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const double eta = (eta_bits & 1) ? -1.0 : 1.0;
    eta_bits += x[mu];
    int xf[4] = {x[0], x[1], x[2], x[3]};
    int xb[4] = {x[0], x[1], x[2], x[3]};
    xf[mu] = (x[mu] + 1 == Ls[mu]) ? 0 : x[mu] + 1;
    xb[mu] = (x[mu] == 0) ? Ls[mu] - 1 : x[mu] - 1;
    const int sf = cb_of(g, xf[0], xf[1], xf[2], xf[3]);
    const int sb = cb_of(g, xb[0], xb[1], xb[2], xb[3]);
    double bf = eta, bb = eta;
    if (mu == 3 && g.ap) {
      if (x[3] == g.L3 - 1) bf = -bf;
      if (x[3] == 0) bb = -bb;
    }
    double u[18], v[6];
    load_link<P64, 0>(links, g.Ve, P, mu, s, u);
    na_load(in, sf, v);
    mv_acc(u, v, bf, acc);
    load_link<P64, 0>(links, g.Ve, 1 - P, mu, sb, u);
    na_load(in, sb, v);
    mvdag_acc(u, v, -bb, acc);
  }
}

// t_odd = D_oe in_even
__global__ void __launch_bounds__(NA_BT) k_na_doe(const Geom g, const void *links, const double2 *in,
                                                  double2 *t) {
  const int s = blockIdx.x * NA_BT + threadIdx.x;
  if (s >= g.Ve) return;
  double acc[6];
  na_hop_sum(g, links, 1, s, in, acc);
  na_store(t, s, acc);
}

// out_even = m4 in - D_eo t; dot = sum Re<in, out> (FP64, fixed-order reduction
// through the static scratch: ticket at offset 0, partials at NA_TICKET_BYTES)
__global__ void __launch_bounds__(NA_BT) k_na_deo_dot(const Geom g, const void *links, double m4,
                                                      const double2 *in, const double2 *t, double2 *out,
                                                      double *dot, unsigned char *scratch) {
  unsigned *ticket = reinterpret_cast<unsigned *>(scratch);
  double *partials = reinterpret_cast<double *>(scratch + NA_TICKET_BYTES);
  const int s = blockIdx.x * NA_BT + threadIdx.x;
  double d = 0.0;
  if (s < g.Ve) {
    double acc[6], c[6], o[6];
    na_hop_sum(g, links, 0, s, t, acc);
    na_load(in, s, c);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      o[i] = m4 * c[i] - acc[i];
      d += c[i] * o[i];
    }
    na_store(out, s, o);
  }
  __shared__ double red[NA_BT / 32];
  __shared__ int am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  d = warp_sum(d);
  if (lane == 0) red[warp] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < NA_BT / 32; ++w) b += red[w];
    partials[blockIdx.x] = b;
    __threadfence();
    am_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double sum = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += NA_BT) sum += __ldcg(partials + i);
  sum = warp_sum(sum);
  if (lane == 0) red[warp] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < NA_BT / 32; ++w) tot += red[w];
    if (dot) *dot = tot;
    *ticket = 0u;
  }
}

// p is device memory of `device` (or managed memory, which every device reaches)
bool na_is_device(const void *p, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == device;
}

}  // namespace

extern "C" int stag_mdagm_dot_noalloc(stag_ctx *ctx, double mass, const double *in_even, double *tmp_odd,
                                      double *out_even, double *dot) {
  if (!ctx) return STAG_ERR_ARG;
  const Geom g = ctx_geom(ctx);
  const int nb = (g.Ve + NA_BT - 1) / NA_BT;
  if (nb > NA_MAX_BLOCKS) {
    ctx_set_error(ctx, "stag_mdagm_dot_noalloc: lattice too large for the fixed scratch "
                       "(at most 8388608 sites per parity)");
    return STAG_ERR_ARG;
  }
  if (!in_even || !tmp_odd || !out_even) {
    ctx_set_error(ctx, "stag_mdagm_dot_noalloc: NULL vector");
    return STAG_ERR_ARG;
  }
  if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) {
    cudaGetLastError();
    ctx_set_error(ctx, "stag_mdagm_dot_noalloc: cudaSetDevice failed");
    return STAG_ERR_CUDA;
  }
  const int dev = ctx_device(ctx);
  if (!na_is_device(in_even, dev) || !na_is_device(tmp_odd, dev) || !na_is_device(out_even, dev) ||
      (dot && !na_is_device(dot, dev))) {
    ctx_set_error(ctx, "stag_mdagm_dot_noalloc: every pointer must be device memory of the context's GPU");
    return STAG_ERR_ARG;
  }
  const void *links = nullptr;
  cudaStream_t st;
  if (ctx_fp64_links(ctx, &links, &st) != STAG_OK) {
    ctx_set_error(ctx, "no gauge field: call stag_links_upload first");
    return STAG_ERR_STATE;
  }
  unsigned char *scratch = nullptr;
  cudaError_t e = na_scratch(dev, &scratch);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) {
    k_na_doe<<<nb, NA_BT, 0, st>>>(g, links, reinterpret_cast<const double2 *>(in_even),
                                   reinterpret_cast<double2 *>(tmp_odd));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_na_deo_dot<<<nb, NA_BT, 0, st>>>(g, links, 4.0 * mass * mass, reinterpret_cast<const double2 *>(in_even),
                                       reinterpret_cast<const double2 *>(tmp_odd),
                                       reinterpret_cast<double2 *>(out_even), dot, scratch);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    ctx_set_error(ctx, cudaGetErrorString(e));
    return STAG_ERR_CUDA;
  }
  return STAG_OK;
}
