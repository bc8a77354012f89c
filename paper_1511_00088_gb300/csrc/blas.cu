// blas.cu -- launchers of the fused BLAS-1 kernels, layout conversions, the
// SU(3) check, and the dispatcher of the half-operator instantiations.
#include "launch.h"

namespace stag {

cudaError_t launch_dslash(int LP, int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                          cudaStream_t st, const DsArgs &a, const void **kptr) {
  switch (LP) {
    case P64: return launch_dslash_p64(recon, VP, OP, NS, EPI, lanes, nblocks, st, a, kptr);
    case P32: return launch_dslash_p32(recon, VP, OP, NS, EPI, lanes, nblocks, st, a, kptr);
    case P16: return launch_dslash_p16(recon, VP, OP, NS, EPI, lanes, nblocks, st, a, kptr);
    case PBF: return launch_dslash_pbf(recon, VP, OP, NS, EPI, lanes, nblocks, st, a, kptr);
  }
  return cudaErrorNotSupported;
}

// (VP, RP) pairs used by the solver: (P64,P64) FP64 CG; (P32,P32), (P16,P32),
// (PBF,P32) mixed precision with FP32 residual and iterate.
#define STAG_BLAS_PAIRS(X, NS_) \
  X(P64, P64, NS_) X(P32, P32, NS_) X(P16, P32, NS_) X(PBF, P32, NS_)

#define STAG_INIT(VP_, RP_, NS_)                                               \
  if (VP == VP_ && RP == RP_ && NS == NS_) {                                   \
    k_cg_init<VP_, RP_, NS_, BLAS_BT><<<nblocks, BLAS_BT, 0, st>>>(a);         \
    return cudaGetLastError();                                                 \
  }

cudaError_t launch_cg_init(int VP, int RP, int NS, int nblocks, cudaStream_t st, const BlasArgs &a) {
  STAG_BLAS_PAIRS(STAG_INIT, 1)
  STAG_BLAS_PAIRS(STAG_INIT, 4)
  STAG_BLAS_PAIRS(STAG_INIT, 8)
  return cudaErrorNotSupported;
}

cudaError_t launch_accum_x(int RP, int NS, int nblocks, cudaStream_t st, const BlasArgs &a) {
#define STAG_ACC(RP_, NS_)                                                     \
  if (RP == RP_ && NS == NS_) {                                                \
    k_accum_x<RP_, NS_, BLAS_BT><<<nblocks, BLAS_BT, 0, st>>>(a);              \
    return cudaGetLastError();                                                 \
  }
  STAG_ACC(P64, 1) STAG_ACC(P64, 4) STAG_ACC(P64, 8)
  STAG_ACC(P32, 1) STAG_ACC(P32, 4) STAG_ACC(P32, 8)
#undef STAG_ACC
  return cudaErrorNotSupported;
}

// grid = nsys blocks of FIN_BT threads; block j reduces system j's nv partial
// arrays of nbx entries each
// Written for latency: every global load is issued before any result is
// used (partials, the system's state), the state is updated in registers and
// stored once, and with a single system there is no cross-block ticket and no
// fence (the next kernel in the stream sees the stores).
__global__ void __launch_bounds__(FIN_BT) k_finalize(const Ctl c, int fin, int nbx, int nv, int nsys,
                                                     const SysState *st_in) {
  constexpr int PER = 4;  // partials per thread per value in flight at once
  __shared__ double red[NVMAX][FIN_BT / 32];
  __shared__ double sums[NVMAX];
  const int j = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  grid_dep_trigger();
  grid_dep_wait();
  SysState st;
  if (threadIdx.x == 0) st = (st_in != nullptr) ? st_in[j] : c.st[j];
  double acc[NVMAX];
#pragma unroll
  for (int v = 0; v < NVMAX; ++v) acc[v] = 0.0;
  for (int base = 0; base < nbx; base += PER * FIN_BT) {
    double x[NVMAX][PER];
#pragma unroll
    for (int v = 0; v < NVMAX; ++v)
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int i = base + u * FIN_BT + threadIdx.x;
        x[v][u] = (v < nv && i < nbx) ? c.partials[((long long)j * NVMAX + v) * c.pstride + i] : 0.0;
      }
#pragma unroll
    for (int v = 0; v < NVMAX; ++v) acc[v] += (x[v][0] + x[v][1]) + (x[v][2] + x[v][3]);
  }
#pragma unroll
  for (int v = 0; v < NVMAX; ++v) {
    const double w = warp_sum(acc[v]);
    if (lane == 0) red[v][warp] = w;
  }
  __syncthreads();
  if (warp < NVMAX) {
    const double w = warp_sum(red[warp][lane]);
    if (lane == 0) sums[warp] = w;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  {
    bool part;
    if (fin == FIN_INIT) part = true;
    else if (fin == FIN_RESID) part = ((st.done == 0 || st.done == 3) && st.update != 0);
    else part = (st.done == 0);
    if (part && fin != FIN_NONE) finalize_system(st, fin, sums);
    if ((part && fin != FIN_NONE) || st_in != nullptr) c.st[j] = st;
  }
  int running = 0, upd = 0;
  if (nsys > 1) {
    __threadfence();
    const unsigned t = atomicAdd(c.all_ticket, 1u);
    if (t != (unsigned)(nsys - 1)) return;
    *c.all_ticket = 0u;
    __threadfence();
    for (int q = 0; q < nsys; ++q) {
      const int done = __ldcg(&c.st[q].done);
      if (done == 0 || done == 3) {
        running = 1;
        if (__ldcg(&c.st[q].update)) upd = 1;
      }
    }
  } else {
    running = (st.done == 0 || st.done == 3) ? 1 : 0;
    upd = running && st.update;
  }
  if (fin == FIN_NORM) {
    // absolute bound on the number of loop passes, whatever the state says
    const int passes = c.flags[2] + 1;
    c.flags[2] = passes;
    if (passes > c.flags[3]) running = 0;
  }
  if (fin == FIN_RESID) c.flags[5] += 1;  // executions of the reliable-update step
  // a CG kernel gave up waiting for its staged links: the iterates are void,
  // so the loop and the update stop here and the host reports the timeout
  if (*(volatile int *)(c.flags + 4) != 0) running = upd = 0;
  c.flags[0] = running;
  c.flags[1] = upd;
  if (c.use_graph_cond) {
    if (fin == FIN_NORM) cudaGraphSetConditional(c.h_update, (unsigned)upd);
    if (fin == FIN_NORM || fin == FIN_RESID) cudaGraphSetConditional(c.h_loop, (unsigned)running);
  }
}

static inline int nblk(long long n, int bt) { return (int)((n + bt - 1) / bt); }

cudaError_t launch_finalize(const Ctl &c, int fin, int nbx, int nv, int nsys, cudaStream_t st, bool pdl,
                            const SysState *st_in) {
  return launch_ex(k_finalize, nsys, FIN_BT, st, pdl, c, fin, nbx, nv, nsys, st_in);
}

cudaError_t launch_pack_vec(int P, const double2 *src, VecArg dst, int k, int Ve, cudaStream_t st) {
  const int nb = nblk(Ve, 256);
  switch (P) {
    case P64: k_pack_vec<P64><<<nb, 256, 0, st>>>(src, dst, k, Ve); break;
    case P32: k_pack_vec<P32><<<nb, 256, 0, st>>>(src, dst, k, Ve); break;
    case P16: k_pack_vec<P16><<<nb, 256, 0, st>>>(src, dst, k, Ve); break;
    case PBF: k_pack_vec<PBF><<<nb, 256, 0, st>>>(src, dst, k, Ve); break;
    default: return cudaErrorNotSupported;
  }
  return cudaGetLastError();
}

__global__ void k_split_full(const double2 *__restrict__ full, VecArg e, VecArg o, int k, Geom g) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.Ve) return;
#pragma unroll
  for (int par = 0; par < 2; ++par) {
    int x[4];
    site_coords(g, par, s, x);
    const long long lex = x[0] + (long long)g.L0 * (x[1] + (long long)g.L1 * (x[2] + (long long)g.L2 * x[3]));
    double v[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 w = full[lex * 3 + c];
      v[2 * c] = w.x;
      v[2 * c + 1] = w.y;
    }
    store_vec<P64>(par == 0 ? e : o, k, s, g.Ve, v);
  }
}

__global__ void k_merge_full(VecArg e, int ke, VecArg o, int ko, double2 *__restrict__ full, Geom g) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.Ve) return;
#pragma unroll
  for (int par = 0; par < 2; ++par) {
    int x[4];
    site_coords(g, par, s, x);
    const long long lex = x[0] + (long long)g.L0 * (x[1] + (long long)g.L1 * (x[2] + (long long)g.L2 * x[3]));
    double v[6];
    load_vec_rw<P64>(par == 0 ? e : o, par == 0 ? ke : ko, s, g.Ve, v);
#pragma unroll
    for (int c = 0; c < 3; ++c) full[lex * 3 + c] = make_double2(v[2 * c], v[2 * c + 1]);
  }
}

cudaError_t launch_split_full(const double2 *full, VecArg e, VecArg o, int k, Geom g, cudaStream_t st) {
  k_split_full<<<nblk(g.Ve, 256), 256, 0, st>>>(full, e, o, k, g);
  return cudaGetLastError();
}

cudaError_t launch_merge_full(VecArg e, int ke, VecArg o, int ko, double2 *full, Geom g, cudaStream_t st) {
  k_merge_full<<<nblk(g.Ve, 256), 256, 0, st>>>(e, ke, o, ko, full, g);
  return cudaGetLastError();
}

cudaError_t launch_unpack_vec(int P, VecArg src, int k, double2 *dst, int Ve, cudaStream_t st) {
  const int nb = nblk(Ve, 256);
  switch (P) {
    case P64: k_unpack_vec<P64><<<nb, 256, 0, st>>>(src, k, dst, Ve); break;
    case P32: k_unpack_vec<P32><<<nb, 256, 0, st>>>(src, k, dst, Ve); break;
    case P16: k_unpack_vec<P16><<<nb, 256, 0, st>>>(src, k, dst, Ve); break;
    case PBF: k_unpack_vec<PBF><<<nb, 256, 0, st>>>(src, k, dst, Ve); break;
    default: return cudaErrorNotSupported;
  }
  return cudaGetLastError();
}

cudaError_t launch_convert_vec(int PIN, int POUT, VecArg src, VecArg dst, int nsys, int Ve,
                               cudaStream_t st) {
  const int nb = nblk((long long)nsys * Ve, 256);
#define STAG_CV(A, B)                                                          \
  if (PIN == A && POUT == B) {                                                 \
    k_convert_vec<A, B><<<nb, 256, 0, st>>>(src, dst, nsys, Ve);               \
    return cudaGetLastError();                                                 \
  }
  STAG_CV(P16, P32) STAG_CV(PBF, P32) STAG_CV(P32, P16) STAG_CV(P32, PBF)
  STAG_CV(P64, P16) STAG_CV(P64, PBF) STAG_CV(P64, P32) STAG_CV(P32, P64)
#undef STAG_CV
  return cudaErrorNotSupported;
}

cudaError_t launch_pack_links_tiled(int LP, int recon, const double2 *src, void *dst, Geom g, int ntile,
                                    cudaStream_t st) {
  const int nb = nblk(16ll * g.Ve, 256);
#define STAG_PLT(P_, R_)                                                        \
  if (LP == P_ && recon == R_) {                                                \
    k_pack_links_tiled<P_, R_><<<nb, 256, 0, st>>>(src, dst, g, ntile);         \
    return cudaGetLastError();                                                  \
  }
  STAG_PLT(P32, 0) STAG_PLT(P32, 1) STAG_PLT(P16, 0) STAG_PLT(P16, 1) STAG_PLT(PBF, 0) STAG_PLT(PBF, 1)
#undef STAG_PLT
  return cudaErrorNotSupported;
}

cudaError_t launch_pack_links(int LP, int recon, const double2 *src, void *dst, Geom g,
                              cudaStream_t st) {
  const long long n = 8ll * g.Ve;  // 4 V links
  const int nb = nblk(n, 256);
#define STAG_PL(A, R)                                                          \
  if (LP == A && recon == R) {                                                 \
    k_pack_links<A, R><<<nb, 256, 0, st>>>(src, dst, g);                       \
    return cudaGetLastError();                                                 \
  }
  STAG_PL(P64, 0) STAG_PL(P32, 0) STAG_PL(P32, 1) STAG_PL(P16, 0) STAG_PL(P16, 1)
  STAG_PL(PBF, 0) STAG_PL(PBF, 1)
#undef STAG_PL
  return cudaErrorNotSupported;
}

// max over links of max(|U U^dag - 1|_max, |det U - 1|), FP64
__global__ void k_su3_defect(const double2 *__restrict__ U, long long nlinks, unsigned long long *out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double d = 0.0;
  if (i < nlinks) {
    double2 u[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = U[i * 9 + e];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        double re = 0.0, im = 0.0;  // (U U^dag)_ab = sum_c U_ac conj(U_bc)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double2 x = u[3 * a + c], y = u[3 * b + c];
          re += x.x * y.x + x.y * y.y;
          im += x.y * y.x - x.x * y.y;
        }
        if (a == b) re -= 1.0;
        d = fmax(d, fmax(fabs(re), fabs(im)));
      }
    // det = u0 (u4 u8 - u5 u7) - u1 (u3 u8 - u5 u6) + u2 (u3 u7 - u4 u6)
    auto mul = [](double2 x, double2 y) { return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); };
    auto sub = [](double2 x, double2 y) { return make_double2(x.x - y.x, x.y - y.y); };
    const double2 c0 = sub(mul(u[4], u[8]), mul(u[5], u[7]));
    const double2 c1 = sub(mul(u[3], u[8]), mul(u[5], u[6]));
    const double2 c2 = sub(mul(u[3], u[7]), mul(u[4], u[6]));
    const double2 t0 = mul(u[0], c0), t1 = mul(u[1], c1), t2 = mul(u[2], c2);
    const double dre = t0.x - t1.x + t2.x - 1.0, dim = t0.y - t1.y + t2.y;
    d = fmax(d, fmax(fabs(dre), fabs(dim)));
    if (!(d == d)) d = 1e300;  // NaN counts as a defect
  }
  // block max, then one atomic per block (non-negative doubles order as uint64)
  __shared__ double sm[256];
  sm[threadIdx.x] = d;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(sm[0]));
}

cudaError_t launch_su3_defect(const double2 *U, long long nlinks, unsigned long long *out,
                              cudaStream_t st) {
  k_su3_defect<<<nblk(nlinks, 256), 256, 0, st>>>(U, nlinks, out);
  return cudaGetLastError();
}

}  // namespace stag
