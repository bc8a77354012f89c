// stag_kernels.cuh -- device code of libstag (sm_103a): the staggered half
// operator D_oe / D_eo with fused epilogues, the fused BLAS-1 steps of CG,
// deterministic FP64 cross-CTA reductions and the reliable-update bookkeeping.
//
// Operator (the one-link staggered operator inside the mixed-precision CG of
// Sec. 3 of the paper; the paper names it without writing it down):
//   (D psi)(x) = sum_mu [ eta_mu(x) b_mu(x) U_mu(x) psi(x+mu)
//                       - eta_mu(x) b_mu(x-mu) U_mu(x-mu)^dag psi(x-mu) ]
//   eta_mu(x) = (-1)^(x_0+...+x_{mu-1}), b_t = -1 on the link from t = Lt-1
//   (antiperiodic time), applied from the coordinates, never folded into U.
//
// Device layouts (structure of arrays, coalesced in the site index s):
//   links  [parity][mu][element e][Ve]  complex (e = 3 row + col; 9, or 6 with
//          reconstruct-12 where row 2 = conj(row0 x row1) is rebuilt in registers)
//   vector [system][colour][Ve] complex; FP16/BF16 vectors add one FP32 scale
//          per site and system: value = code * scale, scale = max |component|.
//   tiled site-owned links (the single-system CG kernels at FP32/FP16/BF16):
//          [parity][tile of LT sites][slot l][element e][LT] complex, slot
//          mu = U_mu(x), slot 4 + mu = U_mu(x - mu) (the backward link, stored
//          again at the site that uses it), so the 8 links of a chunk of sites
//          are one contiguous block, moved into shared memory by one bulk copy.
// One thread owns one output site and NS systems; the 8 links of the site are
// loaded once into registers and applied to all NS systems.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace stag {

enum { P64 = 0, P32 = 1, P16 = 2, PBF = 3 };

template <int P> struct Tr;
template <> struct Tr<P64> { typedef double R; typedef double2 S2; static constexpr bool scaled = false; };
template <> struct Tr<P32> { typedef float R; typedef float2 S2; static constexpr bool scaled = false; };
template <> struct Tr<P16> { typedef float R; typedef __half2 S2; static constexpr bool scaled = true; };
template <> struct Tr<PBF> { typedef float R; typedef __nv_bfloat162 S2; static constexpr bool scaled = true; };

// ---------------------------------------------------------------------------
// plain-old-data argument blocks (passed by value to kernels)
// ---------------------------------------------------------------------------
// Division by a run-time invariant divisor with one multiply-high and shifts
// (Granlund & Montgomery, "Division by invariant integers using
// multiplication", 1994): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// q = (t + ((n - t) >> min(l,1))) >> max(l-1,0) with t = umulhi(m, n); exact
// for every 32-bit n.  Built on the host by make_fastdiv().
struct FastDiv {
  unsigned m, s1, s2;
};

inline FastDiv make_fastdiv(unsigned d) {
  unsigned l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.m = (unsigned)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
  f.s1 = l ? 1u : 0u;
  f.s2 = l ? l - 1 : 0u;
  return f;
}

__device__ __forceinline__ unsigned fast_div(unsigned n, const FastDiv &f) {
  const unsigned t = __umulhi(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

struct Geom {
  int L0, L1, L2, L3;  // Lx, Ly, Lz, Lt
  int Lxh;             // Lx / 2
  int Ve;              // sites per parity
  int ap;              // antiperiodic time boundary
  FastDiv dLxh, dL1, dL2;  // division by Lx/2, Ly, Lz
};

struct VecArg {
  void *v;          // [nsys][3][Ve] complex of the storage type
  float *scale;     // [nsys][Ve] (FP16/BF16 only)
  long long sstr;   // complex elements per system (3 * Ve)
};

// per-system CG state in device memory (FP64 scalars of the mixed CG)
struct SysState {
  double m4;        // 4 m^2
  double bnorm2;    // ||b||^2
  double rho;       // ||r||^2 of the iterated residual
  double pAp;       // <p, A p>
  double alpha, beta;
  double true_res;  // ||b - A x|| / ||b|| at the last reliable update
  double tol;       // stop when ||b - A x|| / ||b|| <= tol
  double delta;     // reliable update when ||r|| < delta * rmax (0: only at tol)
  double rho_prev;  // ||r||^2 one iteration back (beta after a reliable update)
  double pnorm2;    // |p|^2 of the current direction
  double rp;        // Re <r, p> of the current residual and direction
  double rmax2;     // ||r||^2 at the last reliable update
  int maxiter;
  int iter;
  int done;         // 0 running, 3 stopped until the pending FP64 check, 1 converged,
                    // 2 iteration cap, -5 breakdown
  int update;       // a reliable update is pending (run at the end of the unrolled block)
  int n_updates;
  int ref_full;     // 1: bnorm2 holds (2m)^2 |b|^2 of a full-lattice source b (the
                    // even-site source b_s = 2m b_e - D_eo b_o is what the CG solves)
};

struct Ctl {
  SysState *st;          // [nsys]
  double *partials;      // [nsys][NVMAX][pstride]   one per block of the reducing kernel
  unsigned *all_ticket;  // [1] finalize blocks done
  int *flags;            // [0] any system running, [1] any reliable update due,
                         // [2] passes of the norm finalize this solve, [3] cap on [2],
                         // [4] a bulk-copy wait gave up, [5] reliable-update steps run
  int pstride;           // partial slots per (system, value)
  int use_graph_cond;    // call cudaGraphSetConditional on the handles below
  cudaGraphConditionalHandle h_loop, h_update;
};

enum { GATE_NONE = 0, GATE_RUNNING = 1, GATE_UPDATE = 2 };
enum { EPI_PLAIN = 0, EPI_MDAGM = 1, EPI_CG_K1 = 2, EPI_RESID = 3, EPI_CG_K2 = 4, EPI_CG_K1R = 5 };
enum { FIN_NONE = 0, FIN_ALPHA = 1, FIN_NORM = 2, FIN_RESID = 3, FIN_INIT = 4, FIN_ALPHA_R = 5 };

struct DsArgs {
  Geom g;
  int par_out;           // parity of the output sites
  const void *links;     // [2][4][NE][Ve] of the link storage type
  VecArg in;             // input on the other parity (EPI_CG_K1: p_old)
  VecArg center;         // EPI_MDAGM: the vector the mass term multiplies; EPI_RESID: x;
                         // EPI_CG_K2: p (read p_old, written p_new)
  VecArg out;            // output (EPI_RESID: the reduced-precision residual)
  VecArg aux;            // EPI_RESID: the source b (FP64); EPI_CG_K1/K2: the residual r
  VecArg xlo;            // EPI_CG_K2: the partial solution x_lo (read and written)
  VecArg dir;            // EPI_RESID: the direction p at the residual's precision for
                         // Re<r, p> (v == nullptr: not reduced)
  double m4_single;      // 4 m^2 when ctl == nullptr
  double out_scale;      // EPI_MDAGM: out = out_scale (m4 center - D in) when nonzero
  int nsys, ngroups;
  Ctl ctl;               // ctl.st == nullptr: no gating, no reductions
  int gate, fin;
  int pdl;               // launched as a programmatic dependent of the previous kernel
  // Fold (fold != FIN_NONE): the reduction of the previous CG kernel, of kind
  // `fold` (FIN_ALPHA, FIN_ALPHA_R or FIN_NORM) over fold_nv values and
  // fold_nbx partials per system in fold_partials, is finished by every block
  // of this kernel itself, from the states in ctl.st; the first block of each
  // system group stores the new states to st_out.  fold_partials and st_out
  // must not alias ctl.partials and ctl.st.
  int fold, fold_nbx, fold_nv;
  const double *fold_partials;
  SysState *st_out;
  // tma != 0 (single-system CG kernels): the links are read from links_tile
  // (the tiled site-owned copy, ntile tiles per parity): 1 through shared
  // memory (bulk copies), 2 straight into registers
  int tma, ntile;
  const void *links_tile;
  // tma == 1 only: 1 makes every bounded wait for staged links give up at once
  // (the failure path run on purpose: flag, drain, STAG_ERR_TIMEOUT)
  int wait_giveup;
  // host side only (launch attribute): l2_bytes > 0 marks [l2_base, l2_base +
  // l2_bytes) as an L2 access-policy window, a fraction l2_hit of it persisting
  const void *l2_base;
  size_t l2_bytes;
  float l2_hit;
};

// Multi-shift CG: the shifted systems (A_0 + dm4) x_s = b of one source ride
// on the Krylov space of the base system A_0 (the smallest mass).  Shift
// recurrence (exact for r_s = zeta_s r), per base iteration k with the base's
// alpha_k, beta_{k-1}:
//   zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
//                (alpha_k beta_{k-1} (zeta_{k-1} - zeta_k) + zeta_{k-1} alpha_{k-1} (1 + dm4 alpha_k))
//   p_s = zeta_k r_k + beta_{k-1} (zeta_k / zeta_{k-1})^2 p_s;  x_s += alpha_k (zeta_{k+1} / zeta_k) p_s
// with zeta_0 = zeta_{-1} = 1, alpha_{-1} = 1, beta_{-1} = 0, p_s = 0.
struct ShiftState {
  double dm4;         // 4 m_s^2 - 4 m_0^2 (>= 0)
  double zeta, zeta_prev, alpha_prev;
  int active;         // 1 while the shift's recurrence runs
  int iter;           // base iterations it took part in
};

struct MsArgs {
  DsArgs d;           // nsys base systems; ctl.st = their states; the fold of the first CG kernel's sums
  int nsh;            // shifts per base system
  VecArg r;           // base residuals r_k (FP32, [nsys])
  VecArg ps, xs;      // shifted directions and solutions (FP32, [nsys * nsh], slot j * nsh + q)
  ShiftState *sh;     // [nsys * nsh]
  double tol2;        // a shift stops when zeta_{k+1}^2 |r_k|^2 <= tol2 |b|^2
  int nbx;            // blocks per base system
};

struct BlasArgs {
  int Ve;
  VecArg p, r, x, b, x64, t;   // meanings per kernel
  int nsys, ngroups;
  Ctl ctl;
  int gate, fin;
  // k_cg_init of a full-lattice solve (be.v != nullptr): the even and odd
  // halves of the full sources (FP64), source of system j = j / ref_nmass;
  // the reference norm is (2m)^2 (|b_e|^2 + |b_o|^2) instead of |b|^2
  VecArg be, bo;
  int ref_nmass;
};

// ---------------------------------------------------------------------------
// conversions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 to_r2(double2 a) { return a; }
__device__ __forceinline__ float2 to_r2(float2 a) { return a; }
__device__ __forceinline__ float2 to_r2(__half2 a) { return __half22float2(a); }
__device__ __forceinline__ float2 to_r2(__nv_bfloat162 a) { return __bfloat1622float2(a); }

template <int P> __device__ __forceinline__ typename Tr<P>::S2 from_r(typename Tr<P>::R re, typename Tr<P>::R im);
template <> __device__ __forceinline__ double2 from_r<P64>(double re, double im) { return make_double2(re, im); }
template <> __device__ __forceinline__ float2 from_r<P32>(float re, float im) { return make_float2(re, im); }
template <> __device__ __forceinline__ __half2 from_r<P16>(float re, float im) {
  return __halves2half2(__float2half_rn(re), __float2half_rn(im));
}
template <> __device__ __forceinline__ __nv_bfloat162 from_r<PBF>(float re, float im) {
  return __halves2bfloat162(__float2bfloat16_rn(re), __float2bfloat16_rn(im));
}

template <class S2> __device__ __forceinline__ S2 ldg2(const S2 *p) { return __ldg(p); }
template <> __device__ __forceinline__ __half2 ldg2<__half2>(const __half2 *p) {
  unsigned u = __ldg(reinterpret_cast<const unsigned *>(p));
  return *reinterpret_cast<__half2 *>(&u);
}
template <> __device__ __forceinline__ __nv_bfloat162 ldg2<__nv_bfloat162>(const __nv_bfloat162 *p) {
  unsigned u = __ldg(reinterpret_cast<const unsigned *>(p));
  return *reinterpret_cast<__nv_bfloat162 *>(&u);
}

// ---------------------------------------------------------------------------
// vectors
// ---------------------------------------------------------------------------
template <int P, class R>
__device__ __forceinline__ void load_vec(const VecArg &f, int k, int s, int Ve, R (&v)[6]) {
  typedef typename Tr<P>::S2 S2;
  const S2 *p = reinterpret_cast<const S2 *>(f.v) + (long long)k * f.sstr + s;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    auto w = to_r2(ldg2(p + (long long)c * Ve));
    v[2 * c] = (R)w.x;
    v[2 * c + 1] = (R)w.y;
  }
  if (Tr<P>::scaled) {
    const float sc = __ldg(f.scale + (long long)k * Ve + s);
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = (R)((float)v[i] * sc);
  }
}

// coherent (non-ldg) load, for vectors the same kernel also writes
template <int P, class R>
__device__ __forceinline__ void load_vec_rw(const VecArg &f, int k, int s, int Ve, R (&v)[6]) {
  typedef typename Tr<P>::S2 S2;
  const S2 *p = reinterpret_cast<const S2 *>(f.v) + (long long)k * f.sstr + s;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    auto w = to_r2(p[(long long)c * Ve]);
    v[2 * c] = (R)w.x;
    v[2 * c + 1] = (R)w.y;
  }
  if (Tr<P>::scaled) {
    const float sc = f.scale[(long long)k * Ve + s];
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = (R)((float)v[i] * sc);
  }
}

// Store one site.  FP16/BF16: scale = max_i |v_i| (FP32), code_i =
// round-to-nearest-even(v_i / scale) with the quotient correctly rounded in
// FP32; a zero site stores zero codes and scale 0.
template <int P, class R>
__device__ __forceinline__ void store_vec(const VecArg &f, int k, int s, int Ve, const R (&v)[6]) {
  typedef typename Tr<P>::S2 S2;
  typedef typename Tr<P>::R SR;
  S2 *p = reinterpret_cast<S2 *>(f.v) + (long long)k * f.sstr + s;
  if (Tr<P>::scaled) {
    float a[6];
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      a[i] = (float)v[i];
      m = fmaxf(m, fabsf(a[i]));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float qr = 0.f, qi = 0.f;
      if (m > 0.f) {
        qr = __fdiv_rn(a[2 * c], m);
        qi = __fdiv_rn(a[2 * c + 1], m);
      }
      p[(long long)c * Ve] = from_r<P>((SR)qr, (SR)qi);
    }
    f.scale[(long long)k * Ve + s] = m;
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) p[(long long)c * Ve] = from_r<P>((SR)v[2 * c], (SR)v[2 * c + 1]);
  }
}

// Store the share of one site written by `lane` of its LANES lanes: colours
// c with c % LANES == lane; for FP16/BF16 the last lane also writes the
// per-site scale.  Every lane holds the whole site, so the scale (max over the
// 6 components) is computed locally and the codes equal those of store_vec.
template <int P, int LANES, class R>
__device__ __forceinline__ void store_site_share(const VecArg &f, int k, int s, int Ve, int lane,
                                                 const R (&v)[6]) {
  typedef typename Tr<P>::S2 S2;
  typedef typename Tr<P>::R SR;
  S2 *p = reinterpret_cast<S2 *>(f.v) + (long long)k * f.sstr + s;
  if (Tr<P>::scaled) {
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) m = fmaxf(m, fabsf((float)v[i]));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c % LANES != lane) continue;
      float qr = 0.f, qi = 0.f;
      if (m > 0.f) {
        qr = __fdiv_rn((float)v[2 * c], m);
        qi = __fdiv_rn((float)v[2 * c + 1], m);
      }
      p[(long long)c * Ve] = from_r<P>((SR)qr, (SR)qi);
    }
    if (lane == LANES - 1) f.scale[(long long)k * Ve + s] = m;
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c % LANES == lane) p[(long long)c * Ve] = from_r<P>((SR)v[2 * c], (SR)v[2 * c + 1]);
  }
}

// ---------------------------------------------------------------------------
// links
// ---------------------------------------------------------------------------
constexpr int LT = 64;  // sites per tile of the tiled site-owned link layout
constexpr int TMA_STAGES = 2;  // shared-memory stages of the bulk-copied links

// one link from its NE element planes at p, p + stride, ... (SMEM: shared
// memory, else global through the read-only path); row 2 rebuilt for RECON
template <int LP, int RECON, bool SMEM, class R>
__device__ __forceinline__ void load_link_at(const typename Tr<LP>::S2 *p, long long stride, R (&u)[18]) {
  constexpr int NE = RECON ? 6 : 9;
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    auto w = to_r2(SMEM ? p[e * stride] : ldg2(p + e * stride));
    u[2 * e] = (R)w.x;
    u[2 * e + 1] = (R)w.y;
  }
  if (RECON) {
    // row2 = conj(row0 x row1): c0 = conj(a1 b2 - a2 b1), c1 = conj(a2 b0 - a0 b2),
    // c2 = conj(a0 b1 - a1 b0), a = row 0, b = row 1
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int i = (c + 1) % 3, j = (c + 2) % 3;
      const R ar_i = u[2 * i], ai_i = u[2 * i + 1], ar_j = u[2 * j], ai_j = u[2 * j + 1];
      const R br_i = u[6 + 2 * i], bi_i = u[6 + 2 * i + 1], br_j = u[6 + 2 * j], bi_j = u[6 + 2 * j + 1];
      const R re = (ar_i * br_j - ai_i * bi_j) - (ar_j * br_i - ai_j * bi_i);
      const R im = (ar_i * bi_j + ai_i * br_j) - (ar_j * bi_i + ai_j * br_i);
      u[12 + 2 * c] = re;
      u[12 + 2 * c + 1] = -im;
    }
  }
}

template <int LP, int RECON, class R>
__device__ __forceinline__ void load_link(const void *base, int Ve, int par, int mu, int s, R (&u)[18]) {
  typedef typename Tr<LP>::S2 S2;
  constexpr int NE = RECON ? 6 : 9;
  load_link_at<LP, RECON, false>(reinterpret_cast<const S2 *>(base) + (long long)((par * 4 + mu) * NE) * Ve + s,
                                 (long long)Ve, u);
}

// ---------------------------------------------------------------------------
// bulk copies into shared memory (the TMA engine), completed on an mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// orders this thread's earlier shared-memory accesses (and, after a block
// barrier, the block's) before its later bulk copies into shared memory
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// bytes (a multiple of 16; both addresses 16-byte aligned) from global src to
// shared dst; the barrier's current phase completes when they have landed
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait until the phase with parity `parity` of the barrier has completed;
// gives up (false) after about a second (the global timer, checked every 64
// polls) or max_polls polls, whichever comes first (max_polls = 0: gives up
// at once unless nothing is awaited)
constexpr int MBAR_MAX_POLLS = 1 << 20;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, int max_polls = MBAR_MAX_POLLS) {
  const uint32_t b = smem_addr(bar);
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < max_polls; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 63) == 63 && global_ns() - t0 > 1000000000ull) return false;
  }
  return false;
}

// a * b + c, one rounding (FMA) at either precision
__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }

// acc += sgn * (U v).  In FP64 every complex multiply-accumulate is two FMA
// chains per component (re += ur vr - ui vi, im += ur vi + ui vr): 4
// instructions for 8 flops where a*b - c*d + h takes 6, which matters because
// the FP64 operator is bound by GB300's FP64 pipe (~87 % busy).  FP32 keeps
// the expression form: the chains cost the memory-bound FP32 kernels
// registers (123 -> 138 for the second CG kernel, one block fewer per SM).
template <class R>
__device__ __forceinline__ void mv_acc(const R (&u)[18], const R (&v)[6], R sgn, R (&acc)[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R hr = 0, hi = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R ur = u[2 * (3 * a + b)], ui = u[2 * (3 * a + b) + 1];
      if (sizeof(R) == 8) {
        hr = fmar(ur, v[2 * b], hr);
        hr = fmar(-ui, v[2 * b + 1], hr);
        hi = fmar(ur, v[2 * b + 1], hi);
        hi = fmar(ui, v[2 * b], hi);
      } else {
        hr += ur * v[2 * b] - ui * v[2 * b + 1];
        hi += ur * v[2 * b + 1] + ui * v[2 * b];
      }
    }
    acc[2 * a] += sgn * hr;
    acc[2 * a + 1] += sgn * hi;
  }
}

// acc += sgn * (U^dag v)
template <class R>
__device__ __forceinline__ void mvdag_acc(const R (&u)[18], const R (&v)[6], R sgn, R (&acc)[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R hr = 0, hi = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R ur = u[2 * (3 * b + a)], ui = u[2 * (3 * b + a) + 1];
      if (sizeof(R) == 8) {
        hr = fmar(ur, v[2 * b], hr);
        hr = fmar(ui, v[2 * b + 1], hr);
        hi = fmar(ur, v[2 * b + 1], hi);
        hi = fmar(-ui, v[2 * b], hi);
      } else {
        hr += ur * v[2 * b] + ui * v[2 * b + 1];
        hi += ur * v[2 * b + 1] - ui * v[2 * b];
      }
    }
    acc[2 * a] += sgn * hr;
    acc[2 * a + 1] += sgn * hi;
  }
}

#ifndef STAG_FFMA2
#define STAG_FFMA2 0
#endif
#if STAG_FFMA2
// FP32 forms on Blackwell's packed FP32x2 FMA (two lanes of a float2 per
// instruction): with v_b = (re, im), a complex multiply-accumulate is
//   h += Re(U) (v_re, v_im) + Im(U) (-v_im, v_re)       (U v)
//   h += Re(U) (v_re, v_im) + Im(U) ( v_im, -v_re)      (U^dag v)
// two packed FMAs instead of four scalar ones; the swizzled v is formed once
// per colour and reused by the three rows.  Off by default (-DSTAG_FFMA2=1):
// the swizzled copies raise the CG kernels from 117-126 to 126-136 registers,
// past the 128 that keep 4 blocks per SM -- single-source solves gained 1.3 %,
// 16-source solves lost 13 %.
__device__ __forceinline__ float2 bcast2(float x) { return make_float2(x, x); }

__device__ __forceinline__ void mv_acc(const float (&u)[18], const float (&v)[6], float sgn, float (&acc)[6]) {
  float2 vs[3], vw[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    vs[b] = make_float2(v[2 * b], v[2 * b + 1]);
    vw[b] = make_float2(-v[2 * b + 1], v[2 * b]);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 h = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      h = __ffma2_rn(bcast2(u[2 * (3 * a + b)]), vs[b], h);
      h = __ffma2_rn(bcast2(u[2 * (3 * a + b) + 1]), vw[b], h);
    }
    const float2 r = __ffma2_rn(bcast2(sgn), h, make_float2(acc[2 * a], acc[2 * a + 1]));
    acc[2 * a] = r.x;
    acc[2 * a + 1] = r.y;
  }
}

__device__ __forceinline__ void mvdag_acc(const float (&u)[18], const float (&v)[6], float sgn, float (&acc)[6]) {
  float2 vs[3], vd[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    vs[b] = make_float2(v[2 * b], v[2 * b + 1]);
    vd[b] = make_float2(v[2 * b + 1], -v[2 * b]);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 h = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      h = __ffma2_rn(bcast2(u[2 * (3 * b + a)]), vs[b], h);
      h = __ffma2_rn(bcast2(u[2 * (3 * b + a) + 1]), vd[b], h);
    }
    const float2 r = __ffma2_rn(bcast2(sgn), h, make_float2(acc[2 * a], acc[2 * a + 1]));
    acc[2 * a] = r.x;
    acc[2 * a + 1] = r.y;
  }
}
#endif

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
__device__ __forceinline__ void site_coords(const Geom &g, int par, int s, int (&x)[4]) {
  const unsigned q1 = fast_div((unsigned)s, g.dLxh);  // y + Ly (z + Lz t)
  const unsigned q2 = fast_div(q1, g.dL1);            // z + Lz t
  const unsigned q3 = fast_div(q2, g.dL2);            // t
  const int xh = s - (int)q1 * g.Lxh;
  x[1] = (int)q1 - (int)q2 * g.L1;
  x[2] = (int)q2 - (int)q3 * g.L2;
  x[3] = (int)q3;
  x[0] = 2 * xh + ((par + x[1] + x[2] + x[3]) & 1);
}

__device__ __forceinline__ int cb_of(const Geom &g, int x0, int x1, int x2, int x3) {
  return (x0 >> 1) + g.Lxh * (x1 + g.L1 * (x2 + g.L2 * x3));
}

// ---------------------------------------------------------------------------
// deterministic reductions: per-block partials, the last block of a group sums
// them in a fixed order and runs the finaliser of each system of the group;
// the last group to finish publishes the loop/update flags.
// ---------------------------------------------------------------------------
constexpr int NVMAX = 2;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialisation may be scheduled while its predecessor in the stream is still
// running; grid_dep_wait() returns once every predecessor grid has completed
// and its writes are visible (a no-op for an ordinary launch), and nothing
// before it touches memory.  grid_dep_trigger() lets the successor be
// scheduled once every block of this grid has reached it.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// gate of one system by its state (GATE_RUNNING or GATE_UPDATE)
__device__ __forceinline__ bool state_gate(const SysState &s, int gate) {
  if (gate == GATE_RUNNING) return s.done == 0;
  return (s.done == 0 || s.done == 3) && s.update != 0;
}

__device__ __forceinline__ bool sys_gate(const Ctl &c, int gate, int j, int nsys) {
  if (j >= nsys) return false;
  if (gate == GATE_NONE || c.st == nullptr) return true;
  const SysState &s = c.st[j];
  if (gate == GATE_RUNNING) return s.done == 0;
  return (s.done == 0 || s.done == 3) && s.update != 0;
}

// Per-system scalar logic of the CG iteration, run once per reduction by the
// thread that holds the FP64 sums.  Written with few dependent FP64 operations
// (GB300's FP64 pipe is narrow and long-latency): squares are compared
// instead of norms, and square roots are taken only for the reported residual.
//   FIN_ALPHA:   sums |t|^2, |p|^2 of the new direction p = r + beta p_old:
//                alpha = rho / (4 m^2 |p|^2 + |t|^2)  (= <p, A p>, D_eo^dag = -D_oe)
//   FIN_ALPHA_R: as FIN_ALPHA with |p|^2 = rho + 2 beta Re<r, p_old> + beta^2 |p_old|^2
//                (the first kernel then only reduces |t|^2)
//   FIN_NORM:    sums |r|^2, Re<r, p>: beta = rho_new / rho; when |r| < delta
//                r_max (reliable update), |r| <= tol |b| or the iteration cap is
//                reached, an update becomes pending and the system pauses
//                (done = 3) until the FP64 recomputation decides: iterating on
//                past the trigger (up to a pass of 16 iterations) let the FP32
//                recurrences run below their rounding floor on small systems
//   FIN_RESID:   sums of the FP64 recomputation |b - A x|^2, Re<r, p>: converged,
//                capped, or continue with rho = |r_true|^2, beta = rho / rho_prev
//   FIN_INIT:    |b|^2 and |r|^2 of the starting residual
// (breakdown, done = -5, on a non-positive <p, A p> or a non-finite sum)
__device__ __forceinline__ void finalize_system(SysState &s, int fin, const double *sum) {
  if (fin == FIN_ALPHA || fin == FIN_ALPHA_R) {
    const double p2 = (fin == FIN_ALPHA) ? sum[1] : s.rho + s.beta * (2.0 * s.rp + s.beta * s.pnorm2);
    const double pAp = s.m4 * p2 + sum[0];
    s.pnorm2 = p2;
    s.pAp = pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) {
      s.done = -5;
      return;
    }
    s.alpha = s.rho / pAp;
  } else if (fin == FIN_NORM) {
    const double rr = sum[0];
    s.iter += 1;
    if (!isfinite(rr)) {
      s.done = -5;
      return;
    }
    s.rp = sum[1];
    s.rho_prev = s.rho;
    s.beta = rr / s.rho;
    s.rho = rr;
    // convergence candidate, iteration cap or reliable-update trigger: the
    // system pauses (done = 3, its kernels gated off) until the update step at
    // the end of the pass recomputes its residual in FP64 and decides
    if (rr <= s.tol * s.tol * s.bnorm2 || s.iter >= s.maxiter || rr < s.delta * s.delta * s.rmax2) {
      s.update = 1;
      s.done = 3;
    }
  } else if (fin == FIN_RESID) {
    const double rr = sum[0];
    s.update = 0;
    s.n_updates += 1;
    if (!isfinite(rr)) {
      s.done = -5;
      return;
    }
    s.rmax2 = rr;
    s.rp = sum[1];
    if (rr <= s.tol * s.tol * s.bnorm2) {
      s.done = 1;
    } else if (s.iter >= s.maxiter) {
      s.done = 2;
    } else {
      s.done = 0;
      s.beta = rr / s.rho_prev;
      s.rho = rr;
    }
    s.true_res = sqrt(rr / s.bnorm2);
  } else if (fin == FIN_INIT) {
    s.bnorm2 = sum[0];
    s.rho = sum[1];
    s.rho_prev = sum[1];
    s.rmax2 = s.ref_full ? sum[1] : sum[0];
    s.pnorm2 = 0.0;
    s.rp = 0.0;
    s.iter = 0;
    s.update = 0;
    s.n_updates = 0;
    s.alpha = s.beta = s.pAp = 0.0;
    if (sum[0] == 0.0 || (s.ref_full && sum[1] == 0.0)) {  // zero source (x = 0 is exact)
      s.true_res = 0.0;
      s.done = 1;
    } else {
      s.true_res = 1.0;
      s.done = 0;
    }
  }
}

// The previous kernel's reduction, finished inside this kernel (DsArgs::fold):
// every block sums the fold_nbx partials of each of its NS systems in the same
// fixed order (a strided sum per thread, a warp tree, the warps in order) and
// runs the same scalar logic on the same stored state, so all blocks hold
// bit-identical states; the block with bx0 == 0 stores them.  The partials are
// read straight after grid_dep_wait(), in one round of loads per thread.
template <int NS, int BT>
__device__ __forceinline__ void fold_state(const DsArgs &a, int j0, int bx0, SysState *sst) {
  constexpr int NW = BT / 32;
  constexpr int PER = (NS == 1) ? 8 : 1;  // partials per thread and value in flight at once
  __shared__ double red[NS][NVMAX][NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nbx = a.fold_nbx, nv = a.fold_nv;
  const long long ps = a.ctl.pstride;
  double acc[NS][NVMAX];
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int v = 0; v < NVMAX; ++v) acc[k][v] = 0.0;
  for (int base = 0; base < nbx; base += PER * BT) {
    double x[NS][NVMAX][PER];
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int v = 0; v < NVMAX; ++v)
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int i = base + u * BT + (int)threadIdx.x;
          x[k][v][u] = (j0 + k < a.nsys && v < nv && i < nbx)
                           ? a.fold_partials[((long long)(j0 + k) * NVMAX + v) * ps + i]
                           : 0.0;
        }
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int v = 0; v < NVMAX; ++v)
#pragma unroll
        for (int u = 0; u < PER; ++u) acc[k][v] += x[k][v][u];
  }
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int v = 0; v < NVMAX; ++v) {
      const double w = warp_sum(acc[k][v]);
      if (lane == 0) red[k][v][warp] = w;
    }
  __syncthreads();
  if ((int)threadIdx.x < NS) {
    const int k = threadIdx.x, j = j0 + k;
    if (j < a.nsys) {
      double sum[NVMAX];
#pragma unroll
      for (int v = 0; v < NVMAX; ++v) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) t += red[k][v][w];
        sum[v] = t;
      }
      SysState st = a.ctl.st[j];
      if (st.done == 0) finalize_system(st, a.fold, sum);
      sst[k] = st;
      if (bx0 == 0) a.st_out[j] = st;
    }
  }
  __syncthreads();
}

// Reductions, in two stages (both with fixed summation order, so reruns are
// bit-identical):
//  1. block_partials, in every block of a reducing kernel: a 32-lane tree and
//     the warp sums in warp order, in FP32 when T = float (GB300 runs FP64 at
//     a small fraction of the FP32 rate, with long latency); the block sum is
//     stored as one FP64 partial per (system, value) with a plain store -- no
//     fence, no atomic, so no block waits on a memory round trip;
//  2. k_finalize, launched right after on the same stream: one block per
//     system sums that system's partials in block order (FP64), runs the
//     system's scalar logic, and the last finalize block to finish publishes
//     the loop/update flags and the graph conditions.
template <int NS, int NV, class T>
__device__ __forceinline__ void block_partials(const Ctl &c, T (&val)[NS][NV], int j0, int nsys, int bx) {
  __shared__ T red[32][NS * NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T w = warp_sum(val[k][v]);
      if (lane == 0) red[warp][k * NV + v] = w;
    }
  __syncthreads();
  if (threadIdx.x < NS * NV) {
    const int kv = threadIdx.x, k = kv / NV, v = kv % NV;
    T s = 0;
    for (int w = 0; w < nwarp; ++w) s += red[w][kv];
    if (j0 + k < nsys) c.partials[((long long)(j0 + k) * NVMAX + v) * c.pstride + bx] = (double)s;
  }
}

constexpr int FIN_BT = 1024;

// grid = nsys blocks of FIN_BT threads; block j reduces system j's nv partial
// arrays of nbx entries each (defined in blas.cu).  st_in != nullptr: the
// states are read from st_in and all written to c.st (the other buffer of a
// double-buffered pair); else updated in place in c.st.
__global__ void k_finalize(const Ctl c, int fin, int nbx, int nv, int nsys, const SysState *st_in);

// ---------------------------------------------------------------------------
// the half operator with fused epilogues
// ---------------------------------------------------------------------------
// Thread mapping: LANES consecutive lanes own one output site (LANES = 1 or 2);
// a lane handles 4 / LANES directions, and for each direction loads both links
// and both neighbour vectors before using them, so a thread has at most four
// dependent memory rounds (two with LANES = 2) and many loads in flight.  With
// LANES = 2 a butterfly sums the two halves, then the lanes share the stores.
// (Four lanes per site, one direction each, was measured slower: the warp then
// touches 4 widely separated link planes per load and issues 4x the index math.)
//
// EPI_PLAIN:  out = D in
// EPI_MDAGM:  out = m4 center - D in
// EPI_CG_K1:  t = D_oe p_new with p_new = r + beta p_old formed in the gather;
//             |t|^2 and |p_new|^2 per system -> FIN_ALPHA
// EPI_CG_K1R: t = D_oe r + beta t_old (the same t by linearity, one gathered
//             vector instead of two); |t|^2 per system -> FIN_ALPHA_R
// EPI_CG_K2:  p_new (again, at the centre), Ap = m4 p_new - D_eo t,
//             r -= alpha Ap, x_lo += alpha p_new; |r|^2, Re<r,p> -> FIN_NORM
// EPI_RESID:  (FP64) out = b - (m4 x - D in), stored at the output precision,
//             plus ||b - A x||^2 and Re<r, p> per system (FP64) -> FIN_RESID
// __launch_bounds__(BT, 1): without the minimum-blocks argument ptxas caps the
// registers and serialises the loads of the hops; with it, the loads of a
// thread's directions are all in flight together (measured: 27 us instead of
// 34 us for D_oe at 20^3 x 64, FP32).
// (The FP64 kernels are bound by GB300's FP64 pipe and keep 4 blocks per SM.)
// TMA (one system, FP32/FP16/BF16 links) selects where the links come from:
//  0: the plane layout [parity][mu][element][Ve] (the backward links gathered
//     at the neighbours);
//  1: the tiled site-owned copy through a two-stage ring in dynamic shared
//     memory; one thread issues each chunk's bulk copy a round ahead (the first
//     before the wait for the predecessor grid, as the links never change
//     during a solve), so the link stream needs no registers;
//  2: the tiled site-owned copy loaded straight into registers: a warp's 8
//     links then lie in one contiguous block of 32 LT-site rows (fewer DRAM
//     pages per load round than 48 planes of the plane layout).
#ifndef STAG_DS_MINB
#define STAG_DS_MINB 1  // minimum resident blocks per SM asked of ptxas (reduced-precision links)
#endif
template <int LP, int RECON, int VP, int OP, int NS, int EPI, int BT, int LANES, int TMA = 0>
__global__ void __launch_bounds__(BT, LP == P64 ? 4 : STAG_DS_MINB) k_dslash(const DsArgs a) {
  static_assert(!TMA || (NS == 1 && LP != P64), "tiled links: one system, reduced-precision links");
  typedef typename Tr<LP>::R R;
  typedef typename Tr<LP>::S2 LS2;
  constexpr int RP = (LP == P64) ? P64 : P32;  // precision of the residual r
  constexpr bool XPAY_GATHER = (EPI == EPI_CG_K1);  // fold r + beta p into the neighbour gather
  // reduction values per system: K1 |t|^2, |p|^2; K2 |r|^2, Re<r,p>; RESID
  // |b - A x|^2, Re<r,p>; K1R |t|^2
  constexpr int NV = (EPI == EPI_CG_K1 || EPI == EPI_CG_K2 || EPI == EPI_RESID) ? 2 : 1;
  constexpr int DPL = 4 / LANES;  // directions per lane
  // number of centre vectors the epilogue reads at this site
  constexpr int NC = (EPI == EPI_CG_K2) ? 3 : (EPI == EPI_RESID) ? 3 : (EPI == EPI_MDAGM || EPI == EPI_CG_K1R) ? 1 : 0;
  // one system: every load of the site is issued before any arithmetic (one
  // memory round trip per thread); several systems: per direction
  constexpr bool HOIST = (NS == 1);
  const Geom g = a.g;
  const int Ve = g.Ve;
  const int G = a.ngroups;
  const int grp = blockIdx.x % G, bx0 = blockIdx.x / G;
  // The grid may hold fewer blocks than there are chunks of BT / LANES sites
  // (one wave of resident blocks): each block then takes every nbx-th chunk
  // and still leaves one partial per reduced value.
  const int nbx = (int)gridDim.x / G;
  constexpr int SPB = BT / LANES;  // sites per chunk
  const int nchunk = (Ve + SPB - 1) / SPB;
  const int j0 = grp * NS;
  const int lane = LANES == 1 ? 0 : (int)(threadIdx.x % LANES);
  grid_dep_trigger();
  // bulk-copied links: NSTG stages of CHUNK bytes (this block's chunks in turn)
  constexpr int NSTG = TMA_STAGES;
  constexpr int NEL = RECON ? 6 : 9;
  constexpr unsigned CHUNK = (unsigned)(SPB * 8 * NEL * sizeof(LS2));
  extern __shared__ __align__(128) unsigned char stage_mem[];
  __shared__ __align__(8) uint64_t stage_bar[NSTG];
  // a bounded wait of this block gave up, or an earlier kernel's did: no more
  // copies are issued and no thread waits again (the results are void)
  __shared__ volatile int stage_failed;
  const int nmine = bx0 < nchunk ? (nchunk - 1 - bx0) / nbx + 1 : 0;  // chunks of this block
  // Chunk q goes to stage q % NSTG, whose barrier completes phase q / NSTG when
  // it lands.  Chunk q + NSTG is issued only after every thread has waited for
  // chunk q successfully, so each stage has at most one copy outstanding: that
  // of the last chunk issued into it.  `issued` (thread 0) counts the chunks.
  int issued = 0;
  auto issue = [&](int q) {  // bulk copy of this block's chunk q into stage q % NSTG
    const LS2 *src = reinterpret_cast<const LS2 *>(a.links_tile) +
                     ((long long)a.par_out * a.ntile + (long long)(bx0 + q * nbx) * (SPB / LT)) * (8 * NEL * LT);
    bulk_copy_g2s(stage_mem + (q % NSTG) * CHUNK, src, CHUNK, &stage_bar[q % NSTG]);
    issued = q + 1;
  };
  const int wait_polls = a.wait_giveup ? 0 : MBAR_MAX_POLLS;
  if (TMA == 1) {
    if (threadIdx.x == 0) {
      for (int q = 0; q < NSTG; ++q) mbar_init(&stage_bar[q], 1);
      fence_mbar_init();
      stage_failed = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int q = 0; q < NSTG - 1 && q < nmine; ++q) issue(q);
  }
  grid_dep_wait();
  if (TMA == 1) {
    // an earlier kernel of this solve gave up: this one waits for nothing
    if (threadIdx.x == 0 && a.ctl.flags != nullptr && *(volatile int *)(a.ctl.flags + 4) != 0) stage_failed = 1;
    __syncthreads();
  }
  // the systems' states: as stored, or advanced past the previous kernel's
  // reduction by this block (fold)
  __shared__ SysState sst[NS];
  const SysState *S = (a.ctl.st != nullptr) ? a.ctl.st + j0 : nullptr;
  if (a.fold != FIN_NONE) {
    fold_state<NS, BT>(a, j0, bx0, sst);
    S = sst;
  }
  bool act[NS];
  R m4[NS], beta[NS], alpha[NS];
  bool any = false;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const bool in = j0 + k < a.nsys;
    const bool has = S != nullptr && in;
    act[k] = in && (a.gate == GATE_NONE || !has || state_gate(S[k], a.gate));
    any |= act[k];
    m4[k] = (R)(has ? S[k].m4 : a.m4_single);
    beta[k] = (R)(has ? S[k].beta : 0.0);
    alpha[k] = (R)(has ? S[k].alpha : 0.0);
  }
  R part[NS][NV];  // per-thread reduction values (FP32 in the FP32-arithmetic kernels)
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int v = 0; v < NV; ++v) part[k][v] = 0;
  const int P = a.par_out;

  int round = 0;
  for (int bx = bx0; bx < nchunk; bx += nbx, ++round) {
  const LS2 *lsm = nullptr;  // this round's links in shared memory (TMA == 1)
  if (TMA == 1) {
    if (round > 0) __syncthreads();  // every thread is done with the stage read last round
    if (threadIdx.x == 0 && !stage_failed && round + NSTG - 1 < nmine) {
      fence_proxy_async_smem();
      issue(round + NSTG - 1);
    }
    if (!stage_failed && !mbar_wait(&stage_bar[round % NSTG], (unsigned)(round / NSTG) & 1u, wait_polls)) {
      stage_failed = 1;  // this block waits no more; the host reports the error
      if (a.ctl.flags != nullptr) atomicExch(a.ctl.flags + 4, 1);
    }
    lsm = reinterpret_cast<const LS2 *>(stage_mem + (round % NSTG) * CHUNK);
  }
  const int s = bx * SPB + (int)(threadIdx.x / LANES);
  const bool valid = s < Ve;
  R acc[NS][6];
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[k][i] = 0;

  // centre vectors of the single-system epilogue, loaded up front (HOIST)
  R cpre[NC > 0 ? NC : 1][6];
  if (any && valid) {
    if (HOIST && NC > 0) {
      if (EPI == EPI_CG_K2) {
        load_vec_rw<VP>(a.center, j0, s, Ve, cpre[0]);
        load_vec_rw<RP>(a.aux, j0, s, Ve, cpre[NC > 1 ? 1 : 0]);
        load_vec_rw<RP>(a.xlo, j0, s, Ve, cpre[NC > 2 ? 2 : 0]);
      } else if (EPI == EPI_RESID) {
        load_vec<P64>(a.center, j0, s, Ve, cpre[0]);
        load_vec<P64>(a.aux, j0, s, Ve, cpre[NC > 1 ? 1 : 0]);
        if (a.dir.v != nullptr) load_vec<OP>(a.dir, j0, s, Ve, cpre[NC > 2 ? 2 : 0]);
      } else if (EPI == EPI_CG_K1R) {
        load_vec_rw<VP>(a.out, j0, s, Ve, cpre[0]);
      } else {  // EPI_MDAGM
        load_vec<VP>(a.center, j0, s, Ve, cpre[0]);
      }
    }
    int x[4];
    site_coords(g, P, s, x);
    // the two hops of each direction of this lane: neighbour sites and signs
    int sf[DPL], sb[DPL];
    R bf[DPL], bb[DPL];
#pragma unroll
    for (int dd = 0; dd < DPL; ++dd) {
      const int mu = lane * DPL + dd;
      const int Lmu = mu == 0 ? g.L0 : mu == 1 ? g.L1 : mu == 2 ? g.L2 : g.L3;
      int eb = 0;  // x_0 + ... + x_{mu-1}
      if (mu > 0) eb += x[0];
      if (mu > 1) eb += x[1];
      if (mu > 2) eb += x[2];
      const R eta = (eb & 1) ? R(-1) : R(1);
      const int xm = x[mu];
      int xf[4] = {x[0], x[1], x[2], x[3]};
      int xb[4] = {x[0], x[1], x[2], x[3]};
      xf[mu] = (xm + 1 == Lmu) ? 0 : xm + 1;
      xb[mu] = (xm == 0) ? Lmu - 1 : xm - 1;
      sf[dd] = cb_of(g, xf[0], xf[1], xf[2], xf[3]);
      sb[dd] = cb_of(g, xb[0], xb[1], xb[2], xb[3]);
      bf[dd] = eta;
      bb[dd] = eta;
      if (mu == 3 && g.ap) {
        if (xm == g.L3 - 1) bf[dd] = -bf[dd];
        if (xm == 0) bb[dd] = -bb[dd];
      }
    }
    if (HOIST) {
      R uf[DPL][18], ub[DPL][18], vf[DPL][6], vb[DPL][6];
#pragma unroll
      for (int dd = 0; dd < DPL; ++dd) {
        const int mu = lane * DPL + dd;
        if (TMA == 1) {
          const int i = (int)threadIdx.x / LANES;  // site within the chunk
          const LS2 *q = lsm + (i / LT) * (8 * NEL * LT) + i % LT;
          load_link_at<LP, RECON, true>(q + mu * (NEL * LT), LT, uf[dd]);
          load_link_at<LP, RECON, true>(q + (4 + mu) * (NEL * LT), LT, ub[dd]);
        } else if (TMA == 2) {
          const LS2 *q = reinterpret_cast<const LS2 *>(a.links_tile) +
                         ((long long)P * a.ntile + s / LT) * (8 * NEL * LT) + s % LT;
          load_link_at<LP, RECON, false>(q + mu * (NEL * LT), LT, uf[dd]);
          load_link_at<LP, RECON, false>(q + (4 + mu) * (NEL * LT), LT, ub[dd]);
        } else {
          load_link<LP, RECON>(a.links, Ve, P, mu, s, uf[dd]);
          load_link<LP, RECON>(a.links, Ve, 1 - P, mu, sb[dd], ub[dd]);
        }
        load_vec<VP>(a.in, j0, sf[dd], Ve, vf[dd]);
        load_vec<VP>(a.in, j0, sb[dd], Ve, vb[dd]);
      }
      if (XPAY_GATHER) {  // the operator acts on p_new = r + beta p_old, formed here
#pragma unroll
        for (int dd = 0; dd < DPL; ++dd) {
          R rf[6], rb[6];
          load_vec<RP>(a.aux, j0, sf[dd], Ve, rf);
          load_vec<RP>(a.aux, j0, sb[dd], Ve, rb);
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            vf[dd][i] = rf[i] + beta[0] * vf[dd][i];
            vb[dd][i] = rb[i] + beta[0] * vb[dd][i];
          }
          // |p_new|^2 over the even sites: each even site is the forward-x
          // neighbour of exactly one odd site, so count it there
          if (lane * DPL + dd == 0 && NV > 1) {
            R q = 0;
#pragma unroll
            for (int i = 0; i < 6; ++i) q += vf[dd][i] * vf[dd][i];
            part[0][NV - 1] += q;
          }
        }
      }
#pragma unroll
      for (int dd = 0; dd < DPL; ++dd) {
        mv_acc(uf[dd], vf[dd], bf[dd], acc[0]);
        mvdag_acc(ub[dd], vb[dd], -bb[dd], acc[0]);
      }
    } else {
#pragma unroll
      for (int dd = 0; dd < DPL; ++dd) {
        const int mu = lane * DPL + dd;
        R uf[18], ub[18];
        load_link<LP, RECON>(a.links, Ve, P, mu, s, uf);
        load_link<LP, RECON>(a.links, Ve, 1 - P, mu, sb[dd], ub);
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          if (!act[k]) continue;
          R vf[6], vb[6];
          load_vec<VP>(a.in, k + j0, sf[dd], Ve, vf);
          load_vec<VP>(a.in, k + j0, sb[dd], Ve, vb);
          if (XPAY_GATHER) {
            R rf[6], rb[6];
            load_vec<RP>(a.aux, k + j0, sf[dd], Ve, rf);
            load_vec<RP>(a.aux, k + j0, sb[dd], Ve, rb);
#pragma unroll
            for (int i = 0; i < 6; ++i) {
              vf[i] = rf[i] + beta[k] * vf[i];
              vb[i] = rb[i] + beta[k] * vb[i];
            }
            if (mu == 0 && NV > 1) {
              R q = 0;
#pragma unroll
              for (int i = 0; i < 6; ++i) q += vf[i] * vf[i];
              part[k][NV - 1] += q;
            }
          }
          mv_acc(uf, vf, bf[dd], acc[k]);
          mvdag_acc(ub, vb, -bb[dd], acc[k]);
        }
      }
    }
  }
  if (LANES > 1) {
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int o = 1; o < LANES; o <<= 1) acc[k][i] += __shfl_xor_sync(0xffffffffu, acc[k][i], o);
  }

  // The epilogue loop runs on every lane (act[] is uniform across the block) so
  // that the warp barriers are reached by all lanes; per-lane work is
  // predicated on `valid`.
  if (any) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (!act[k]) continue;
      const int j = k + j0;
      if (EPI == EPI_CG_K2) {
        // p_new = r + beta p_old at this site (the first kernel formed the same at
        // the neighbours); Ap = 4 m^2 p_new - D_eo t; r -= alpha Ap; x_lo += alpha
        // p_new; p_new, r, x_lo stored; |r|^2 and Re<r, p_new> reduced.  Ap itself
        // is never stored.
        R cv[6], rv[6], xv[6];
        if (valid) {
          if (HOIST) {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
              cv[i] = cpre[0][i];
              rv[i] = cpre[NC > 1 ? 1 : 0][i];
              xv[i] = cpre[NC > 2 ? 2 : 0][i];
            }
          } else {
            load_vec_rw<VP>(a.center, j, s, Ve, cv);
            load_vec_rw<RP>(a.aux, j, s, Ve, rv);
            load_vec_rw<RP>(a.xlo, j, s, Ve, xv);
          }
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            cv[i] = rv[i] + beta[k] * cv[i];
            const R ap = m4[k] * cv[i] - acc[k][i];
            rv[i] -= alpha[k] * ap;
            xv[i] += alpha[k] * cv[i];
          }
          R q = 0, rp = 0;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            if (c % LANES == lane) {
              q += rv[2 * c] * rv[2 * c] + rv[2 * c + 1] * rv[2 * c + 1];
              rp += rv[2 * c] * cv[2 * c] + rv[2 * c + 1] * cv[2 * c + 1];
            }
          part[k][0] += q;
          part[k][1] += rp;
        }
        if (LANES > 1) __syncwarp();  // every lane has read the site before any lane writes it
        if (valid) {
          store_site_share<VP, LANES>(a.center, j, s, Ve, lane, cv);
          store_site_share<RP, LANES>(a.aux, j, s, Ve, lane, rv);
          store_site_share<RP, LANES>(a.xlo, j, s, Ve, lane, xv);
        }
        continue;
      }
      if (EPI == EPI_CG_K1R) {
        // t = D_oe r + beta t_old (= D_oe (r + beta p_old) by linearity); |t|^2
        R tv[6];
        if (valid) {
          if (HOIST) {
#pragma unroll
            for (int i = 0; i < 6; ++i) tv[i] = cpre[0][i];
          } else {
            load_vec_rw<VP>(a.out, j, s, Ve, tv);
          }
#pragma unroll
          for (int i = 0; i < 6; ++i) tv[i] = acc[k][i] + beta[k] * tv[i];
          R q = 0;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            if (c % LANES == lane) q += tv[2 * c] * tv[2 * c] + tv[2 * c + 1] * tv[2 * c + 1];
          part[k][0] += q;
        }
        if (LANES > 1) __syncwarp();
        if (valid) store_site_share<VP, LANES>(a.out, j, s, Ve, lane, tv);
        continue;
      }
      if (!valid) continue;
      R o[6];
      if (EPI == EPI_PLAIN || EPI == EPI_CG_K1) {
#pragma unroll
        for (int i = 0; i < 6; ++i) o[i] = acc[k][i];
        if (EPI == EPI_CG_K1) {  // |t|^2 over the odd sites
          R q = 0;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            if (c % LANES == lane) q += o[2 * c] * o[2 * c] + o[2 * c + 1] * o[2 * c + 1];
          part[k][0] += q;
        }
      } else if (EPI == EPI_MDAGM) {
        R cv[6];
        if (HOIST) {
#pragma unroll
          for (int i = 0; i < 6; ++i) cv[i] = cpre[0][i];
        } else {
          load_vec<VP>(a.center, j, s, Ve, cv);
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) o[i] = m4[k] * cv[i] - acc[k][i];
        if (a.out_scale != 0.0) {
#pragma unroll
          for (int i = 0; i < 6; ++i) o[i] *= (R)a.out_scale;
        }
      } else {  // EPI_RESID (R = double)
        R xx[6], bv[6];
        R pv[6] = {0, 0, 0, 0, 0, 0};
        if (HOIST) {
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            xx[i] = cpre[0][i];
            bv[i] = cpre[NC > 1 ? 1 : 0][i];
            if (a.dir.v != nullptr) pv[i] = cpre[NC > 2 ? 2 : 0][i];
          }
        } else {
          load_vec<P64>(a.center, j, s, Ve, xx);
          load_vec<P64>(a.aux, j, s, Ve, bv);
          if (a.dir.v != nullptr) load_vec<OP>(a.dir, j, s, Ve, pv);
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) o[i] = bv[i] - (m4[k] * xx[i] - acc[k][i]);
        // Re<r, p> of the residual as it will be stored (rounded to OP)
        typename Tr<OP>::R orr[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) orr[i] = (typename Tr<OP>::R)o[i];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (c % LANES == lane) {
            part[k][0] += o[2 * c] * o[2 * c] + o[2 * c + 1] * o[2 * c + 1];
            part[k][1] += (R)orr[2 * c] * pv[2 * c] + (R)orr[2 * c + 1] * pv[2 * c + 1];
          }
      }
      store_site_share<OP, LANES>(a.out, j, s, Ve, lane, o);
    }
  }
  }  // chunks
  if (TMA == 1) {
    __syncthreads();  // every thread's stage_failed visible: the branch below is uniform
    if (stage_failed) {
      // the copy still outstanding in each stage (that of the last chunk
      // issued into it) lands before the block exits: a wait on its phase,
      // bounded again (the results of this launch are void in any case)
      if (threadIdx.x == 0)
        for (int q = issued - NSTG > 0 ? issued - NSTG : 0; q < issued; ++q)
          mbar_wait(&stage_bar[q % NSTG], (unsigned)(q / NSTG) & 1u);
      __syncthreads();
    }
  }

  if (EPI == EPI_CG_K1 || EPI == EPI_CG_K1R || EPI == EPI_CG_K2 || EPI == EPI_RESID) {
    if (a.ctl.st != nullptr) block_partials<NS, NV>(a.ctl, part, j0, a.nsys, bx0);
  }
}

// ---------------------------------------------------------------------------
// the two CG kernels for several systems, the links shared in shared memory
// ---------------------------------------------------------------------------
// A block of NSW warps (NSW = 4 or 8) owns NSW systems j0 .. j0 + NSW - 1 and
// takes chunks of 32 output sites.  The 8 links of a chunk's sites go into
// shared memory once for all NSW systems (NSW = 4: warp w copies the forward
// and the backward link of direction w; NSW = 8: warp w link slot w), with the
// neighbour sites and signs of the slot; warp w then applies them to system
// j0 + w, one lane per site.  The link loads, the row-2 rebuild and the index
// arithmetic are so paid once per NSW systems, without holding a site's links
// in registers for all of them.  Two buffers: while a chunk is computed, the
// next chunk's links arrive by asynchronous copies (cp.async, no registers),
// and each chunk's gathered vectors are loaded before the barriers that make
// its links ready.  FP32 links and vectors; epilogues EPI_CG_K1R and EPI_CG_K2
// exactly as in k_dslash (one lane per site); reductions per warp.
template <int LP, int RECON, int NSW, int EPI>
__global__ void __launch_bounds__(32 * NSW, 1) k_dslash_mrhs(const DsArgs a) {
  static_assert(LP == P32 && (NSW == 4 || NSW == 8) && (EPI == EPI_CG_K1R || EPI == EPI_CG_K2),
                "FP32, 4 or 8 systems per block, the two CG kernels");
  typedef float R;
  constexpr int BT = 32 * NSW;
  constexpr int NV = (EPI == EPI_CG_K2) ? 2 : 1;
  const Geom g = a.g;
  const int Ve = g.Ve;
  const int G = a.ngroups;
  const int grp = blockIdx.x % G, bx0 = blockIdx.x / G;
  const int nbx = (int)gridDim.x / G;
  const int nchunk = (Ve + 31) / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j0 = grp * NSW, j = j0 + w;
  const int P = a.par_out;
  constexpr int NEL = RECON ? 6 : 9;  // stored complex elements per link
  __shared__ __align__(16) float2 su[2][8][9][32];  // [buffer][slot][element][site]
  __shared__ int snb[2][8][32];                      // neighbour site of the slot
  __shared__ float ssg[2][8][32];                    // its sign (minus for backward hops)
  grid_dep_trigger();
  grid_dep_wait();
  __shared__ SysState sst[NSW];
  const SysState *S = (a.ctl.st != nullptr) ? a.ctl.st + j0 : nullptr;
  if (a.fold != FIN_NONE) {
    fold_state<NSW, BT>(a, j0, bx0, sst);
    S = sst;
  }
  const bool in = j < a.nsys;
  const bool has = S != nullptr && in;
  const bool act = in && (a.gate == GATE_NONE || !has || state_gate(S[w], a.gate));
  const R m4 = (R)(has ? S[w].m4 : a.m4_single);
  const R beta = (R)(has ? S[w].beta : 0.0);
  const R alpha = (R)(has ? S[w].alpha : 0.0);
  R part[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) part[v] = 0;
  typedef typename Tr<LP>::S2 LS2;
  const LS2 *lk = reinterpret_cast<const LS2 *>(a.links);

  // this warp's slots of chunk bx into buffer b: indices, signs, and the
  // stored link elements by asynchronous copies (one commit group per call)
  auto stage = [&](int bx, int b) {
    const int s = bx * 32 + lane;
    if (s < Ve) {
      int x[4];
      site_coords(g, P, s, x);
#pragma unroll
      for (int q = 0; q < 8 / NSW; ++q) {
        const int slot = (NSW == 4) ? (q == 0 ? w : 4 + w) : w;
        const int mu = slot & 3;
        const bool fwd = slot < 4;
        const int Lmu = mu == 0 ? g.L0 : mu == 1 ? g.L1 : mu == 2 ? g.L2 : g.L3;
        int eb = 0;  // x_0 + ... + x_{mu-1}
        if (mu > 0) eb += x[0];
        if (mu > 1) eb += x[1];
        if (mu > 2) eb += x[2];
        R sg = (eb & 1) ? R(-1) : R(1);
        const int xm = x[mu];
        int xn[4] = {x[0], x[1], x[2], x[3]};
        xn[mu] = fwd ? ((xm + 1 == Lmu) ? 0 : xm + 1) : ((xm == 0) ? Lmu - 1 : xm - 1);
        const int sn = cb_of(g, xn[0], xn[1], xn[2], xn[3]);
        if (mu == 3 && g.ap && (fwd ? (xm == g.L3 - 1) : (xm == 0))) sg = -sg;
        snb[b][slot][lane] = sn;
        ssg[b][slot][lane] = fwd ? sg : -sg;
        const LS2 *src = lk + (long long)(((fwd ? P : 1 - P) * 4 + mu) * NEL) * Ve + (fwd ? s : sn);
#pragma unroll
        for (int e = 0; e < NEL; ++e)
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(&su[b][slot][e][lane])),
                       "l"(src + (long long)e * Ve)
                       : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  if (bx0 < nchunk) stage(bx0, 0);
  int b = 0;
  for (int bx = bx0; bx < nchunk; bx += nbx, b ^= 1) {
    const int s = bx * 32 + lane;
    const bool valid = s < Ve;
    __syncthreads();  // buffer b's indices visible; nobody still reads buffer b ^ 1
    // this chunk's gathered and centre vectors, in flight across the barriers below
    R vn[8][6], c0[6], c1[6], c2[6];
    if (act && valid) {
#pragma unroll
      for (int slot = 0; slot < 8; ++slot) load_vec<P32>(a.in, j, snb[b][slot][lane], Ve, vn[slot]);
      if (EPI == EPI_CG_K2) {
        load_vec_rw<P32>(a.center, j, s, Ve, c0);
        load_vec_rw<P32>(a.aux, j, s, Ve, c1);
        load_vec_rw<P32>(a.xlo, j, s, Ve, c2);
      } else {
        load_vec_rw<P32>(a.out, j, s, Ve, c0);
      }
    }
    if (bx + nbx < nchunk) stage(bx + nbx, b ^ 1);
    else asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // this thread's copies of chunk bx
    __syncthreads();                                      // everybody's
    if (RECON && valid) {
      // row 2 = conj(row0 x row1) for this warp's slots, in place
#pragma unroll
      for (int q = 0; q < 8 / NSW; ++q) {
        const int slot = (NSW == 4) ? (q == 0 ? w : 4 + w) : w;
        float2 r0[3], r1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          r0[c] = su[b][slot][c][lane];
          r1[c] = su[b][slot][3 + c][lane];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int i1 = (c + 1) % 3, i2 = (c + 2) % 3;
          const float re = (r0[i1].x * r1[i2].x - r0[i1].y * r1[i2].y) - (r0[i2].x * r1[i1].x - r0[i2].y * r1[i1].y);
          const float im = (r0[i1].x * r1[i2].y + r0[i1].y * r1[i2].x) - (r0[i2].x * r1[i1].y + r0[i2].y * r1[i1].x);
          su[b][slot][6 + c][lane] = make_float2(re, -im);
        }
      }
    }
    if (RECON) __syncthreads();
    if (!(act && valid)) continue;
    R acc[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int slot = 0; slot < 8; ++slot) {
      R u[18];
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        const float2 v2 = su[b][slot][e][lane];
        u[2 * e] = v2.x;
        u[2 * e + 1] = v2.y;
      }
      if (slot < 4) mv_acc(u, vn[slot], ssg[b][slot][lane], acc);
      else mvdag_acc(u, vn[slot], ssg[b][slot][lane], acc);
    }
    if (EPI == EPI_CG_K2) {
      // p_new = r + beta p_old; Ap = 4 m^2 p_new - D_eo t; r -= alpha Ap; x_lo += alpha p_new
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        c0[i] = c1[i] + beta * c0[i];
        const R ap = m4 * c0[i] - acc[i];
        c1[i] -= alpha * ap;
        c2[i] += alpha * c0[i];
      }
      R q = 0, rp = 0;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        q += c1[i] * c1[i];
        rp += c1[i] * c0[i];
      }
      part[0] += q;
      part[NV - 1] += rp;
      store_vec<P32>(a.center, j, s, Ve, c0);
      store_vec<P32>(a.aux, j, s, Ve, c1);
      store_vec<P32>(a.xlo, j, s, Ve, c2);
    } else {
      // t = D_oe r + beta t_old; |t|^2
      R q = 0;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        c0[i] = acc[i] + beta * c0[i];
        q += c0[i] * c0[i];
      }
      part[0] += q;
      store_vec<P32>(a.out, j, s, Ve, c0);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");  // none outstanding at exit
  // one warp per system: its 32-lane sum is the block's partial
  if (a.ctl.st != nullptr) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R t = warp_sum(part[v]);
      if (lane == 0 && in) a.ctl.partials[((long long)j * NVMAX + v) * a.ctl.pstride + bx0] = (double)t;
    }
  }
}

// ---------------------------------------------------------------------------
// fused BLAS-1 steps of the CG iteration (one thread per site, NS systems)
// ---------------------------------------------------------------------------
// reliable update, part 1: x64 += x_lo; x_lo = 0 (systems with an update due)
template <int RP, int NS, int BT>
__global__ void __launch_bounds__(BT) k_accum_x(const BlasArgs a) {
  typedef typename Tr<RP>::R R;
  const int G = a.ngroups, grp = blockIdx.x % G, bx = blockIdx.x / G;
  const int j0 = grp * NS, Ve = a.Ve;
  const int s = bx * BT + threadIdx.x;
  if (s >= Ve) return;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int j = j0 + k;
    if (!sys_gate(a.ctl, a.gate, j, a.nsys)) continue;
    R xl[6];
    double x6[6];
    load_vec_rw<RP>(a.x, j, s, Ve, xl);
    load_vec_rw<P64>(a.x64, j, s, Ve, x6);
    const R z[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 6; ++i) x6[i] += (double)xl[i];
    store_vec<P64>(a.x64, j, s, Ve, x6);
    store_vec<RP>(a.x, j, s, Ve, z);
  }
}

// CG start: x64 = 0, x_lo = 0, r = round(b), p_old = 0 (with beta = 0 the
// first half operator forms p = r); partials ||b||^2 (FP64), ||r||^2 -> FIN_INIT
template <int VP, int RP, int NS, int BT>
__global__ void __launch_bounds__(BT) k_cg_init(const BlasArgs a) {
  typedef typename Tr<RP>::R R;
  const int G = a.ngroups, grp = blockIdx.x % G, bx = blockIdx.x / G;
  const int j0 = grp * NS, Ve = a.Ve;
  const int s = bx * BT + threadIdx.x;
  double part[NS][2];
#pragma unroll
  for (int k = 0; k < NS; ++k) part[k][0] = part[k][1] = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int j = j0 + k;
    if (j >= a.nsys || s >= Ve) continue;
    double b[6];
    load_vec<P64>(a.b, j, s, Ve, b);
    double bb = 0.0;
    R r[6];
    const double z64[6] = {0, 0, 0, 0, 0, 0};
    const R z[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      bb += b[i] * b[i];
      r[i] = (R)b[i];
    }
    store_vec<RP>(a.r, j, s, Ve, r);
    R rr_[6];
    load_vec_rw<RP>(a.r, j, s, Ve, rr_);  // the values the iteration sees
    R rr = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) rr += rr_[i] * rr_[i];
    // p_old = 0, t_old = 0 and beta = 0: the first iteration forms p = r itself
    store_vec<VP>(a.p, j, s, Ve, z);
    store_vec<VP>(a.t, j, s, Ve, z);
    store_vec<RP>(a.x, j, s, Ve, z);
    store_vec<P64>(a.x64, j, s, Ve, z64);
    if (a.be.v != nullptr) {  // full-lattice source: (2m)^2 |b_full|^2 at this site pair
      double e[6], o[6];
      load_vec<P64>(a.be, j / a.ref_nmass, s, Ve, e);
      load_vec<P64>(a.bo, j / a.ref_nmass, s, Ve, o);
      double q = 0.0;
#pragma unroll
      for (int i = 0; i < 6; ++i) q += e[i] * e[i] + o[i] * o[i];
      bb = a.ctl.st[j].m4 * q;
    }
    part[k][0] = bb;
    part[k][1] = (double)rr;
  }
  block_partials<NS, 2>(a.ctl, part, j0, a.nsys, bx);
}

// ---------------------------------------------------------------------------
// layout conversion between the ABI's [Ve][3] FP64 complex and the device SoA
// ---------------------------------------------------------------------------
template <int P>
__global__ void k_pack_vec(const double2 *__restrict__ src, VecArg dst, int k, int Ve) {
  typedef typename Tr<P>::R R;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Ve) return;
  R v[6];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double2 w = src[(long long)s * 3 + c];
    v[2 * c] = (R)w.x;
    v[2 * c + 1] = (R)w.y;
  }
  store_vec<P>(dst, k, s, Ve, v);
}

template <int P>
__global__ void k_unpack_vec(VecArg src, int k, double2 *__restrict__ dst, int Ve) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Ve) return;
  double v[6];
  {
    typename Tr<P>::R w[6];
    load_vec_rw<P>(src, k, s, Ve, w);
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = (double)w[i];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) dst[(long long)s * 3 + c] = make_double2(v[2 * c], v[2 * c + 1]);
}

// full-lattice ABI vector [V][3] (lexicographic sites) <-> its even and odd
// halves (system k of e / o, FP64 device layout); one thread per
// checkerboard index s, which is one even and one odd site
__global__ void k_split_full(const double2 *__restrict__ full, VecArg e, VecArg o, int k, Geom g);
__global__ void k_merge_full(VecArg e, int ke, VecArg o, int ko, double2 *__restrict__ full, Geom g);

// dst = src re-stored at another precision (FP16/BF16 quantise per site)
template <int PIN, int POUT>
__global__ void k_convert_vec(VecArg src, VecArg dst, int nsys, int Ve) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nsys * Ve) return;
  const int k = (int)(i / Ve), s = (int)(i % Ve);
  typename Tr<POUT>::R v[6];
  load_vec_rw<PIN>(src, k, s, Ve, v);
  store_vec<POUT>(dst, k, s, Ve, v);
}

// canonical [4][V][3][3] FP64 links -> [2][4][NE][Ve] at precision LP
// (FP16/BF16 links are stored unscaled: |U_ij| <= 1 for SU(3))
template <int LP, int RECON>
__global__ void k_pack_links(const double2 *__restrict__ src, void *dst, Geom g) {
  typedef typename Tr<LP>::S2 S2;
  typedef typename Tr<LP>::R R;
  constexpr int NE = RECON ? 6 : 9;
  const long long V = 2ll * g.Ve;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // over 4 V links
  if (i >= 4 * V) return;
  const int mu = (int)(i / V);
  const long long lex = i % V;
  int x0 = (int)(lex % g.L0);
  long long r = lex / g.L0;
  const int x1 = (int)(r % g.L1);
  r /= g.L1;
  const int x2 = (int)(r % g.L2);
  const int x3 = (int)(r / g.L2);
  const int par = (x0 + x1 + x2 + x3) & 1;
  const int s = (int)(lex >> 1);
  S2 *d = reinterpret_cast<S2 *>(dst) + (long long)((par * 4 + mu) * NE) * g.Ve + s;
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const double2 w = src[i * 9 + e];
    R re, im;
    if (LP == P64) {
      re = (R)w.x;
      im = (R)w.y;
    } else {
      // FP64 -> FP32 first; FP16/BF16 round that FP32 value
      re = (R)__double2float_rn(w.x);
      im = (R)__double2float_rn(w.y);
    }
    d[(long long)e * g.Ve] = from_r<LP>(re, im);
  }
}

// tiled site-owned copy of the links (see the layout notes at the top): one
// thread per (parity, site, slot); dst zeroed beforehand (the tail of the last
// tiles stays zero); ntile tiles per parity
template <int LP, int RECON>
__global__ void k_pack_links_tiled(const double2 *__restrict__ src, void *dst, Geom g, int ntile) {
  typedef typename Tr<LP>::S2 S2;
  typedef typename Tr<LP>::R R;
  constexpr int NE = RECON ? 6 : 9;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // over 2 Ve 8
  if (i >= 16ll * g.Ve) return;
  const int l = (int)(i & 7);
  const long long ps = i >> 3;
  const int par = (int)(ps / g.Ve), s = (int)(ps % g.Ve);
  int x[4];
  site_coords(g, par, s, x);
  const int mu = l & 3;
  if (l >= 4) {  // the backward link U_mu(x - mu) lives at the neighbour
    const int Lmu = mu == 0 ? g.L0 : mu == 1 ? g.L1 : mu == 2 ? g.L2 : g.L3;
    x[mu] = (x[mu] == 0) ? Lmu - 1 : x[mu] - 1;
  }
  const long long lex = x[0] + (long long)g.L0 * (x[1] + (long long)g.L1 * (x[2] + (long long)g.L2 * x[3]));
  const double2 *w = src + ((long long)mu * 2 * g.Ve + lex) * 9;
  S2 *d = reinterpret_cast<S2 *>(dst) + (((long long)par * ntile + s / LT) * 8 + l) * NE * LT + s % LT;
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    // FP64 -> FP32 first; FP16/BF16 round that FP32 value (as k_pack_links)
    const R re = (R)__double2float_rn(w[e].x), im = (R)__double2float_rn(w[e].y);
    d[(long long)e * LT] = from_r<LP>(re, im);
  }
}

// unitarity and determinant defect of every link -> max into *out (as bits of a
// non-negative double, so an integer atomicMax orders them)
__global__ void k_su3_defect(const double2 *__restrict__ U, long long nlinks, unsigned long long *out);

}  // namespace stag
