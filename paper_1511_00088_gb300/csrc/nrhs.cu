// nrhs.cu -- the two CG kernels for several systems on one lattice (the
// multi-source / multi-mass batches of Sec. 3's workloads), with every link
// loaded once per block and reused by all systems.
//
// A block owns chunks of LT = 64 output sites (one tile of the tiled
// site-owned link copy: the 8 links of each site, forward and backward, in one
// contiguous block) and SL threads per site.  Per chunk:
//   * one bulk copy (cp.async.bulk, mbarrier completion, bounded wait) brings
//     the tile's links into shared memory, the next tile's copy in flight
//     while this one is computed (two stages); with reconstruct-12 the block
//     first rebuilds row 2 of every link once into a full 3x3 copy;
//   * each thread computes its site's coordinates, neighbour indices and
//     staggered/boundary signs once, then loops over the systems j = lane,
//     lane + SL, ...: it gathers the 8 neighbour vectors of system j, applies
//     the links from shared memory and runs the system's epilogue with its
//     own alpha, beta, 4 m^2 (states read once per launch into shared memory).
// The links and the index arithmetic are so paid once per chunk instead of
// once per system (the one-system-per-block form reloads them, from L2, for
// every system).  FP32 links and vectors; epilogues EPI_CG_K1R and EPI_CG_K2
// as in k_dslash.  Reductions: per system a 32-lane tree per warp after each
// chunk, the warp sums in shared memory, one FP64 partial per system and
// block at the end (k_finalize sums them).
#include "launch.h"

namespace stag {

constexpr int NRHS_MAX = 64;  // systems per launch

// dynamic shared memory: two stages of one tile's stored links, plus (reconstruct-12) the full copy
inline unsigned nrhs_smem_bytes(int recon) {
  const unsigned tile = 8u * (recon ? 6u : 9u) * (unsigned)LT * 8u;
  return 2u * tile + (recon ? 8u * 9u * (unsigned)LT * 8u : 0u);
}

template <int RECON, int EPI, int SL>
__global__ void __launch_bounds__(LT * SL, 2) k_cg_nrhs(const DsArgs a) {
  static_assert(EPI == EPI_CG_K1R || EPI == EPI_CG_K2, "the two CG kernels");
  constexpr int BT = LT * SL;
  constexpr int NW = BT / 32;
  constexpr int NEL = RECON ? 6 : 9;
  constexpr int NV = (EPI == EPI_CG_K2) ? 2 : 1;
  constexpr unsigned TILE = 8u * NEL * LT * 8u;  // bytes of one tile's stored links
  extern __shared__ __align__(128) unsigned char smem[];
  float2 *stage0 = reinterpret_cast<float2 *>(smem);
  float2 *full = reinterpret_cast<float2 *>(smem + 2 * TILE);  // [slot][9][LT] (reconstruct-12)
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ volatile int failed;
  __shared__ SysState sst[NRHS_MAX];
  __shared__ float red[NRHS_MAX][NW][NV];
  const Geom g = a.g;
  const int Ve = g.Ve, P = a.par_out, nsys = a.nsys;
  const int tid = threadIdx.x, i = tid % LT, lane = tid / LT, warp = tid >> 5;
  const int ntile = (Ve + LT - 1) / LT;
  const int nmine = (int)blockIdx.x < ntile ? (ntile - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  int issued = 0;  // thread 0: tiles whose copy was issued
  auto issue = [&](int q) {
    const int t = (int)blockIdx.x + q * (int)gridDim.x;
    const float2 *src = reinterpret_cast<const float2 *>(a.links_tile) + ((long long)P * a.ntile + t) * (8 * NEL * LT);
    bulk_copy_g2s(smem + (q & 1) * TILE, src, TILE, &bar[q & 1]);
    issued = q + 1;
  };
  grid_dep_trigger();
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    failed = 0;
  }
  __syncthreads();
  if (tid == 0 && nmine > 0) issue(0);  // the links never change during a solve
  grid_dep_wait();
  for (int j = tid; j < nsys; j += BT) sst[j] = a.ctl.st[j];
  for (int k = tid; k < NRHS_MAX * NW * NV; k += BT) (&red[0][0][0])[k] = 0.f;
  if (tid == 0 && a.ctl.flags != nullptr && *(volatile int *)(a.ctl.flags + 4) != 0) failed = 1;
  __syncthreads();

  for (int round = 0; round < nmine; ++round) {
    const int t = (int)blockIdx.x + round * (int)gridDim.x;
    const float2 *stg = stage0 + (round & 1) * (TILE / 8);
    if (!failed && !mbar_wait(&bar[round & 1], (unsigned)(round >> 1) & 1u)) {
      failed = 1;
      if (a.ctl.flags != nullptr) atomicExch(a.ctl.flags + 4, 1);
    }
    const float2 *L = stg;
    constexpr int LNE = RECON ? 9 : NEL;  // elements per link in the copy the compute reads
    if (RECON) {
      __syncthreads();  // every thread is done with last round's full copy
      // rebuild: 8 LT links, row 2 = conj(row0 x row1)
      for (int k = tid; k < 8 * LT; k += BT) {
        const int slot = k / LT, ii = k % LT;
        const float2 *sp = stg + slot * (NEL * LT) + ii;
        float2 *dp = full + slot * (9 * LT) + ii;
        float2 r0[3], r1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          r0[c] = sp[c * LT];
          r1[c] = sp[(3 + c) * LT];
          dp[c * LT] = r0[c];
          dp[(3 + c) * LT] = r1[c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
          const float re = (r0[c1].x * r1[c2].x - r0[c1].y * r1[c2].y) - (r0[c2].x * r1[c1].x - r0[c2].y * r1[c1].y);
          const float im = (r0[c1].x * r1[c2].y + r0[c1].y * r1[c2].x) - (r0[c2].x * r1[c1].y + r0[c2].y * r1[c1].x);
          dp[(6 + c) * LT] = make_float2(re, -im);
        }
      }
      L = full;
    }
    __syncthreads();  // this round's links ready; last round's stage free
    if (tid == 0 && !failed && round + 1 < nmine) {
      fence_proxy_async_smem();
      issue(round + 1);
    }
    const int s = t * LT + i;
    const bool valid = s < Ve;
    int sf[4], sb[4];
    float bf[4], bb[4];
    if (valid) {
      int x[4];
      site_coords(g, P, s, x);
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        const int Lmu = mu == 0 ? g.L0 : mu == 1 ? g.L1 : mu == 2 ? g.L2 : g.L3;
        int eb = 0;
        if (mu > 0) eb += x[0];
        if (mu > 1) eb += x[1];
        if (mu > 2) eb += x[2];
        const float eta = (eb & 1) ? -1.f : 1.f;
        const int xm = x[mu];
        int xf[4] = {x[0], x[1], x[2], x[3]};
        int xb[4] = {x[0], x[1], x[2], x[3]};
        xf[mu] = (xm + 1 == Lmu) ? 0 : xm + 1;
        xb[mu] = (xm == 0) ? Lmu - 1 : xm - 1;
        sf[mu] = cb_of(g, xf[0], xf[1], xf[2], xf[3]);
        sb[mu] = cb_of(g, xb[0], xb[1], xb[2], xb[3]);
        bf[mu] = eta;
        bb[mu] = eta;
        if (mu == 3 && g.ap) {
          if (xm == g.L3 - 1) bf[mu] = -bf[mu];
          if (xm == 0) bb[mu] = -bb[mu];
        }
      }
    }
    for (int j = lane; j < nsys; j += SL) {
      const SysState &S = sst[j];
      if (!(a.gate == GATE_NONE || state_gate(S, a.gate))) continue;  // uniform per warp
      const float beta = (float)S.beta, alpha = (float)S.alpha, m4 = (float)S.m4;
      float q0 = 0.f, q1 = 0.f;
      if (valid) {
        float vf[4][6], vb[4][6], c0[6], c1[6], c2[6];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          load_vec<P32>(a.in, j, sf[mu], Ve, vf[mu]);
          load_vec<P32>(a.in, j, sb[mu], Ve, vb[mu]);
        }
        if (EPI == EPI_CG_K2) {
          load_vec_rw<P32>(a.center, j, s, Ve, c0);
          load_vec_rw<P32>(a.aux, j, s, Ve, c1);
          load_vec_rw<P32>(a.xlo, j, s, Ve, c2);
        } else {
          load_vec_rw<P32>(a.out, j, s, Ve, c0);
        }
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          float u[18];
          load_link_at<P32, 0, true>(L + mu * (LNE * LT) + i, LT, u);
          mv_acc(u, vf[mu], bf[mu], acc);
          load_link_at<P32, 0, true>(L + (4 + mu) * (LNE * LT) + i, LT, u);
          mvdag_acc(u, vb[mu], -bb[mu], acc);
        }
        if (EPI == EPI_CG_K2) {
          // p = r + beta p_old; A p = 4 m^2 p - D_eo t; r -= alpha A p; x_lo += alpha p
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            c0[k] = c1[k] + beta * c0[k];
            const float ap = m4 * c0[k] - acc[k];
            c1[k] -= alpha * ap;
            c2[k] += alpha * c0[k];
            q0 += c1[k] * c1[k];
            q1 += c1[k] * c0[k];
          }
          store_vec<P32>(a.center, j, s, Ve, c0);
          store_vec<P32>(a.aux, j, s, Ve, c1);
          store_vec<P32>(a.xlo, j, s, Ve, c2);
        } else {
          // t = D_oe r + beta t_old
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            c0[k] = acc[k] + beta * c0[k];
            q0 += c0[k] * c0[k];
          }
          store_vec<P32>(a.out, j, s, Ve, c0);
        }
      }
      q0 = warp_sum(q0);
      if (NV > 1) q1 = warp_sum(q1);
      if ((tid & 31) == 0) {
        red[j][warp][0] += q0;
        if (NV > 1) red[j][warp][NV - 1] += q1;
      }
    }
  }
  __syncthreads();
  if (failed) {
    // the copies still outstanding land before the block exits (bounded)
    if (tid == 0)
      for (int q = issued - 2 > 0 ? issued - 2 : 0; q < issued; ++q) mbar_wait(&bar[q & 1], (unsigned)(q >> 1) & 1u);
    __syncthreads();
  }
  // one FP64 partial per system and value: the warps of the system's lane in order
  if (a.ctl.st != nullptr) {
    for (int k = tid; k < nsys * NV; k += BT) {
      const int j = k / NV, v = k % NV, ln = j % SL;
      float sum = 0.f;
#pragma unroll
      for (int w = 0; w < LT / 32; ++w) sum += red[j][ln * (LT / 32) + w][v];
      a.ctl.partials[((long long)j * NVMAX + v) * a.ctl.pstride + blockIdx.x] = (double)sum;
    }
  }
}

template <int RC_, int EPI_, int SL_>
static cudaError_t nrhs_one(int nblocks, cudaStream_t st, const DsArgs &a, const void **kptr) {
  auto k = k_cg_nrhs<RC_, EPI_, SL_>;
  const unsigned smem = nrhs_smem_bytes(RC_);
  static bool attr_set = false;  // benign race: setting it twice is harmless
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (kptr) {
    *kptr = (const void *)k;
    return cudaSuccess;
  }
  return launch_ex_full(k, nblocks, LT * SL_, smem, st, a.pdl != 0, a.l2_base, a.l2_bytes, a.l2_hit, a);
}

cudaError_t launch_cg_nrhs(int recon, int sl, int EPI, int nblocks, cudaStream_t st, const DsArgs &a,
                           const void **kptr) {
#define STAG_NR(RC_, EPI_, SL_) \
  if (recon == RC_ && EPI == EPI_ && sl == SL_) return nrhs_one<RC_, EPI_, SL_>(nblocks, st, a, kptr);
  STAG_NR(0, EPI_CG_K1R, 2) STAG_NR(0, EPI_CG_K2, 2) STAG_NR(1, EPI_CG_K1R, 2) STAG_NR(1, EPI_CG_K2, 2)
  STAG_NR(0, EPI_CG_K1R, 4) STAG_NR(0, EPI_CG_K2, 4) STAG_NR(1, EPI_CG_K1R, 4) STAG_NR(1, EPI_CG_K2, 4)
#undef STAG_NR
  return cudaErrorNotSupported;
}

unsigned cg_nrhs_smem(int recon) { return nrhs_smem_bytes(recon); }

}  // namespace stag
