// nrhs.cu -- the two CG kernels for several systems on one lattice (the
// multi-source / multi-mass batches of Sec. 3's workloads), with every link
// loaded once per block and reused by all systems.
//
// A block owns chunks of LT = 64 output sites (one tile of the tiled
// site-owned link copy: the 8 links of each site, forward and backward, in one
// contiguous block) and SL threads per site.  Per chunk:
//   * one bulk copy (cp.async.bulk, mbarrier completion, bounded wait) brings
//     the tile's links into shared memory, the next tile's copy in flight
//     while this one is computed (two stages);
//   * each thread computes its site's coordinates, neighbour indices and
//     staggered/boundary signs once; with reconstruct-12 (and in the
//     one-stage form) the block then writes a full 3x3 copy of every link
//     once, row 2 rebuilt, the hop's sign folded in and the backward links
//     stored daggered, so that all 8 hops are one product form;
//   * the SL lanes of a site (lane l: whole warps of 32 consecutive sites)
//     share out the systems still iterating (compacted once per launch): each
//     gathers the 8 neighbour vectors of its system (or, JJ = 2, of two
//     systems in two phases), applies the links from shared memory and runs
//     the system's epilogue with its own alpha, beta, 4 m^2 (states read once
//     per launch into shared memory).
// The links and the index arithmetic are so paid once per chunk instead of
// once per system (the one-system-per-block form reloads them, from L2, for
// every system).  FP32 links and vectors; epilogues EPI_CG_K1R and EPI_CG_K2
// as in k_dslash.  Reductions: per system a 32-lane tree per warp after each
// chunk, the warp sums in shared memory, one FP64 partial per system and
// block at the end (k_finalize sums them).
#include "launch.h"

namespace stag {

constexpr int NRHS_MAX = 64;  // systems per launch

// The SU(3) x colour-vector products on Blackwell's packed FP32x2 FMA.  On the
// stored links (plain links, two stages, no full copy), with v_b = (re, im)
// and w_b = (-im, re), a complex multiply-accumulate is
//   h += Re(U_ab) v_b + Im(U_ab) w_b                      (U v)
//   h += Re(U_ba) v_b - Im(U_ba) w_b                      (U^dag v)
// two packed FMAs instead of four scalar ones, then acc += sign h.  On the full
// copy (signs and daggers folded in) mv_split below needs no sign step and
// no w_b.
__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }

// acc += sgn U v
__device__ __forceinline__ void mv_x2(const float2 *u, int ls, const float2 (&v)[3], float sgn, float2 (&acc)[3]) {
  float2 w[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) w[b] = make_float2(-v[b].y, v[b].x);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 h = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float2 e = u[(3 * a + b) * ls];
      h = __ffma2_rn(bc2(e.x), v[b], h);
      h = __ffma2_rn(bc2(e.y), w[b], h);
    }
    acc[a] = __ffma2_rn(bc2(sgn), h, acc[a]);
  }
}

// acc += sgn U^dag v
__device__ __forceinline__ void mvdag_x2(const float2 *u, int ls, const float2 (&v)[3], float sgn, float2 (&acc)[3]) {
  float2 w[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) w[b] = make_float2(v[b].y, -v[b].x);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 h = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float2 e = u[(3 * b + a) * ls];
      h = __ffma2_rn(bc2(e.x), v[b], h);
      h = __ffma2_rn(bc2(e.y), w[b], h);
    }
    acc[a] = __ffma2_rn(bc2(sgn), h, acc[a]);
  }
}

// acc1 += U (Re v), acc2 += U (Im v), element pairs (Re U_ab, Im U_ab) times
// the broadcast real / imaginary part of v_b: (U v)_a = (acc1.x - acc2.y,
// acc1.y + acc2.x).  The links of the block's full copy already carry the
// site's staggered sign and, for the backward hops, the dagger, so every hop is
// this one form and the two sums combine once per site and system.
__device__ __forceinline__ void mv_split(const float2 *u, int ls, const float2 (&v)[3], float2 (&acc1)[3],
                                         float2 (&acc2)[3]) {
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const float2 vr = bc2(v[b].x), vi = bc2(v[b].y);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float2 e = u[(3 * a + b) * ls];
      acc1[a] = __ffma2_rn(e, vr, acc1[a]);
      acc2[a] = __ffma2_rn(e, vi, acc2[a]);
    }
  }
}

// mv_split for two systems at once: each link element read from shared memory
// serves both
__device__ __forceinline__ void mv_split2(const float2 *u, int ls, const float2 (&va)[3], const float2 (&vb)[3],
                                          float2 (&a1)[3], float2 (&a2)[3], float2 (&b1)[3], float2 (&b2)[3]) {
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const float2 vra = bc2(va[b].x), via = bc2(va[b].y), vrb = bc2(vb[b].x), vib = bc2(vb[b].y);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float2 e = u[(3 * a + b) * ls];
      a1[a] = __ffma2_rn(e, vra, a1[a]);
      a2[a] = __ffma2_rn(e, via, a2[a]);
      b1[a] = __ffma2_rn(e, vrb, b1[a]);
      b2[a] = __ffma2_rn(e, vib, b2[a]);
    }
  }
}

// the three colours of site s of system k (FP32 vector, read-only path)
__device__ __forceinline__ void ld3(const VecArg &f, int k, int s, int Ve, float2 (&v)[3]) {
  const float2 *p = reinterpret_cast<const float2 *>(f.v) + (long long)k * f.sstr + s;
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = __ldg(p + (long long)c * Ve);
}
__device__ __forceinline__ void ld3_rw(const VecArg &f, int k, int s, int Ve, float2 (&v)[3]) {
  const float2 *p = reinterpret_cast<const float2 *>(f.v) + (long long)k * f.sstr + s;
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = p[(long long)c * Ve];
}
__device__ __forceinline__ void st3(const VecArg &f, int k, int s, int Ve, const float2 (&v)[3]) {
  float2 *p = reinterpret_cast<float2 *>(f.v) + (long long)k * f.sstr + s;
#pragma unroll
  for (int c = 0; c < 3; ++c) p[(long long)c * Ve] = v[c];
}

// per-system scalars of a launch, converted once per block
struct SysF {
  float alpha, beta, m4;
  int act;
};

// dynamic shared memory: STG stages of one tile's stored links, plus the full
// 3x3 copy the compute reads (reconstruct-12, or every single-stage form)
inline unsigned nrhs_smem_bytes(int recon, int stg) {
  const unsigned tile = 8u * (recon ? 6u : 9u) * (unsigned)LT * 8u, full = 8u * 9u * (unsigned)LT * 8u;
  return (unsigned)stg * tile + ((recon || stg == 1) ? full : 0u);
}

// STG = 2: two stages, the next tile's copy in flight during the whole round
// (2 blocks per SM); STG = 1: one stage, refilled as soon as this round's
// links are in the full copy (less shared memory: 3 blocks per SM)
// JJ = 2 (reconstruct-12 only): two systems per pass through the thread, in
// two phases (the forward neighbours of both, then the backward ones, so that
// as many loads are in flight as with one system), each link element read
// from shared memory once for both systems
template <int RECON, int EPI, int SL, int STG, int JJ>
__global__ void __launch_bounds__(LT * SL, STG == 1 ? 3 : 2) k_cg_nrhs(const DsArgs a) {
  static_assert(EPI == EPI_CG_K1R || EPI == EPI_CG_K2, "the two CG kernels");
  static_assert(STG == 1 || STG == 2, "one or two stages");
  static_assert(JJ == 1 || (JJ == 2 && (RECON || STG == 1)), "two systems per pass need the full copy");
  constexpr int BT = LT * SL;
  constexpr int NW = BT / 32;
  constexpr int NEL = RECON ? 6 : 9;
  constexpr int NV = (EPI == EPI_CG_K2) ? 2 : 1;
  constexpr bool EXPAND = RECON || STG == 1;  // the compute reads the full copy
  constexpr unsigned TILE = 8u * NEL * LT * 8u;  // bytes of one tile's stored links
  extern __shared__ __align__(128) unsigned char smem[];
  float2 *stage0 = reinterpret_cast<float2 *>(smem);
  float2 *full = reinterpret_cast<float2 *>(smem + STG * TILE);  // [slot][9][LT]
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ volatile int failed;
  __shared__ SysF sf32[NRHS_MAX];
  __shared__ float red[NRHS_MAX][NW][NV];
  __shared__ int act_list[NRHS_MAX];  // the systems this launch updates, in order
  __shared__ int n_act;
  __shared__ float hop_sgn[EXPAND ? 8 : 1][LT];  // the signs the full copy folds in
  const Geom g = a.g;
  const int Ve = g.Ve, P = a.par_out, nsys = a.nsys;
  // lane l = threads [l LT, (l + 1) LT): whole warps, 32 consecutive sites each
  const int tid = threadIdx.x, i = tid % LT, lane = tid / LT, warp = tid >> 5;
  const int ntile = (Ve + LT - 1) / LT;
  const int nmine = (int)blockIdx.x < ntile ? (ntile - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  int issued = 0;  // thread 0: tiles whose copy was issued
  // tile q goes to stage q % STG; its barrier completes phase q / STG when it lands
  auto issue = [&](int q) {
    const int t = (int)blockIdx.x + q * (int)gridDim.x;
    const float2 *src = reinterpret_cast<const float2 *>(a.links_tile) + ((long long)P * a.ntile + t) * (8 * NEL * LT);
    bulk_copy_g2s(smem + (q % STG) * TILE, src, TILE, &bar[q % STG]);
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
  for (int j = tid; j < nsys; j += BT) {
    const SysState S = a.ctl.st[j];
    SysF f;
    f.alpha = (float)S.alpha;
    f.beta = (float)S.beta;
    f.m4 = (float)S.m4;
    f.act = (a.gate == GATE_NONE || state_gate(S, a.gate)) ? 1 : 0;
    sf32[j] = f;
  }
  for (int k = tid; k < NRHS_MAX * NW * NV; k += BT) (&red[0][0][0])[k] = 0.f;
  if (tid == 0 && a.ctl.flags != nullptr && *(volatile int *)(a.ctl.flags + 4) != 0) failed = 1;
  __syncthreads();
  // the active systems, compacted (read after the first round's barrier): the
  // lanes share out only systems that still iterate, so a lane whose systems
  // converged first does not leave its warps idle while the others work
  if (tid == 0) {
    int n = 0;
    for (int j = 0; j < nsys; ++j)
      if (sf32[j].act) act_list[n++] = j;
    n_act = n;
  }

  for (int round = 0; round < nmine; ++round) {
    const int t = (int)blockIdx.x + round * (int)gridDim.x;
    const float2 *stg = stage0 + (round % STG) * (TILE / 8);
    if (!failed && !mbar_wait(&bar[round % STG], (unsigned)(round / STG) & 1u)) {
      failed = 1;
      if (a.ctl.flags != nullptr) atomicExch(a.ctl.flags + 4, 1);
    }
    // this thread's site: neighbour indices and the hop signs (staggered
    // phase, antiperiodic t boundary; backward hops enter with a minus sign)
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
    const float2 *L = stg;  // the stage itself (no full copy: plain links, two stages)
    if (EXPAND) {
      if (lane == 0) {
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          hop_sgn[mu][i] = valid ? bf[mu] : 0.f;
          hop_sgn[4 + mu][i] = valid ? -bb[mu] : 0.f;
        }
      }
      __syncthreads();  // every thread is done with last round's full copy; the signs are in
      // the full copy: sign x link (forward hops), sign x link^dag (backward
      // hops), with (reconstruct-12) row 2 = conj(row0 x row1) rebuilt first
      for (int k = tid; k < 8 * LT; k += BT) {
        const int slot = k / LT, ii = k % LT;
        const float sg = hop_sgn[slot][ii];
        const float2 *sp = stg + slot * (NEL * LT) + ii;
        float2 *dp = full + slot * (9 * LT) + ii;
        float2 m[9];
#pragma unroll
        for (int e = 0; e < NEL; ++e) m[e] = sp[e * LT];
        if (RECON) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
            const float2 *r0 = m, *r1 = m + 3;
            const float re =
                (r0[c1].x * r1[c2].x - r0[c1].y * r1[c2].y) - (r0[c2].x * r1[c1].x - r0[c2].y * r1[c1].y);
            const float im =
                (r0[c1].x * r1[c2].y + r0[c1].y * r1[c2].x) - (r0[c2].x * r1[c1].y + r0[c2].y * r1[c1].x);
            m[6 + c] = make_float2(re, -im);
          }
        }
        if (slot < 4) {
#pragma unroll
          for (int e = 0; e < 9; ++e) dp[e * LT] = make_float2(sg * m[e].x, sg * m[e].y);
        } else {
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) dp[(3 * a + b) * LT] = make_float2(sg * m[3 * b + a].x, -sg * m[3 * b + a].y);
        }
      }
    }
    __syncthreads();  // this round's links ready; the stage the next copy fills is free
    if (tid == 0 && !failed && round + 1 < nmine) {
      fence_proxy_async_smem();
      issue(round + 1);
    }
    const int nact = n_act;
    if constexpr (JJ == 2) {
      for (int k0 = 0; k0 < nact; k0 += 2 * SL) {
        const int ka = k0 + 2 * lane;
        const bool hasA = ka < nact, hasB = ka + 1 < nact;  // uniform per warp
        const int ja = hasA ? act_list[ka] : 0, jb = hasB ? act_list[ka + 1] : 0;
        float qa0 = 0.f, qa1 = 0.f, qb0 = 0.f, qb1 = 0.f;
        if (hasA && valid) {
          const float2 z = make_float2(0.f, 0.f);
          float2 pa1[3] = {z, z, z}, pa2[3] = {z, z, z}, pb1[3] = {z, z, z}, pb2[3] = {z, z, z};
#pragma unroll
          for (int h = 0; h < 2; ++h) {  // forward hops, then backward hops
            float2 va[4][3], vb2[4][3];
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
              const int nb = h == 0 ? sf[mu] : sb[mu];
              ld3(a.in, ja, nb, Ve, va[mu]);
              if (hasB) {
                ld3(a.in, jb, nb, Ve, vb2[mu]);
              } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) vb2[mu][c] = z;
              }
            }
#pragma unroll
            for (int mu = 0; mu < 4; ++mu)
              mv_split2(full + (4 * h + mu) * (9 * LT) + i, LT, va[mu], vb2[mu], pa1, pa2, pb1, pb2);
          }
          float2 accA[3], accB[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            accA[c] = make_float2(pa1[c].x - pa2[c].y, pa1[c].y + pa2[c].x);
            accB[c] = make_float2(pb1[c].x - pb2[c].y, pb1[c].y + pb2[c].x);
          }
          const SysF SA = sf32[ja], SB = sf32[jb];
          if (EPI == EPI_CG_K2) {
            float2 pA[3], rA[3], xA[3], pB[3], rB[3], xB[3];
            ld3_rw(a.center, ja, s, Ve, pA);
            ld3_rw(a.aux, ja, s, Ve, rA);
            ld3_rw(a.xlo, ja, s, Ve, xA);
            if (hasB) {
              ld3_rw(a.center, jb, s, Ve, pB);
              ld3_rw(a.aux, jb, s, Ve, rB);
              ld3_rw(a.xlo, jb, s, Ve, xB);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              pA[k] = __ffma2_rn(bc2(SA.beta), pA[k], rA[k]);
              const float2 ap = __ffma2_rn(bc2(SA.m4), pA[k], make_float2(-accA[k].x, -accA[k].y));
              rA[k] = __ffma2_rn(bc2(-SA.alpha), ap, rA[k]);
              xA[k] = __ffma2_rn(bc2(SA.alpha), pA[k], xA[k]);
              qa0 += rA[k].x * rA[k].x + rA[k].y * rA[k].y;
              qa1 += rA[k].x * pA[k].x + rA[k].y * pA[k].y;
            }
            st3(a.center, ja, s, Ve, pA);
            st3(a.aux, ja, s, Ve, rA);
            st3(a.xlo, ja, s, Ve, xA);
            if (hasB) {
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                pB[k] = __ffma2_rn(bc2(SB.beta), pB[k], rB[k]);
                const float2 ap = __ffma2_rn(bc2(SB.m4), pB[k], make_float2(-accB[k].x, -accB[k].y));
                rB[k] = __ffma2_rn(bc2(-SB.alpha), ap, rB[k]);
                xB[k] = __ffma2_rn(bc2(SB.alpha), pB[k], xB[k]);
                qb0 += rB[k].x * rB[k].x + rB[k].y * rB[k].y;
                qb1 += rB[k].x * pB[k].x + rB[k].y * pB[k].y;
              }
              st3(a.center, jb, s, Ve, pB);
              st3(a.aux, jb, s, Ve, rB);
              st3(a.xlo, jb, s, Ve, xB);
            }
          } else {
            float2 tA[3], tB[3];
            ld3_rw(a.out, ja, s, Ve, tA);
            if (hasB) ld3_rw(a.out, jb, s, Ve, tB);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              tA[k] = __ffma2_rn(bc2(SA.beta), tA[k], accA[k]);
              qa0 += tA[k].x * tA[k].x + tA[k].y * tA[k].y;
            }
            st3(a.out, ja, s, Ve, tA);
            if (hasB) {
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                tB[k] = __ffma2_rn(bc2(SB.beta), tB[k], accB[k]);
                qb0 += tB[k].x * tB[k].x + tB[k].y * tB[k].y;
              }
              st3(a.out, jb, s, Ve, tB);
            }
          }
        }
        qa0 = warp_sum(qa0);
        qb0 = warp_sum(qb0);
        if (NV > 1) {
          qa1 = warp_sum(qa1);
          qb1 = warp_sum(qb1);
        }
        if ((tid & 31) == 0) {
          if (hasA) {
            red[ja][warp][0] += qa0;
            if (NV > 1) red[ja][warp][NV - 1] += qa1;
          }
          if (hasB) {
            red[jb][warp][0] += qb0;
            if (NV > 1) red[jb][warp][NV - 1] += qb1;
          }
        }
      }
    } else {
      for (int k0 = 0; k0 < nact; k0 += SL) {
        const bool has = k0 + lane < nact;  // uniform per warp
        const int j = has ? act_list[k0 + lane] : 0;
        const SysF S = sf32[j];
        const float beta = S.beta, alpha = S.alpha, m4 = S.m4;
        float q0 = 0.f, q1 = 0.f;
        if (has && valid) {
          float2 vf[4][3], vb[4][3], c0[3], c1[3], c2[3];
  #pragma unroll
          for (int mu = 0; mu < 4; ++mu) {
            ld3(a.in, j, sf[mu], Ve, vf[mu]);
            ld3(a.in, j, sb[mu], Ve, vb[mu]);
          }
          if (EPI == EPI_CG_K2) {
            ld3_rw(a.center, j, s, Ve, c0);
            ld3_rw(a.aux, j, s, Ve, c1);
            ld3_rw(a.xlo, j, s, Ve, c2);
          } else {
            ld3_rw(a.out, j, s, Ve, c0);
          }
          float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
          if (EXPAND) {
            float2 acc2[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  #pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
              mv_split(full + mu * (9 * LT) + i, LT, vf[mu], acc, acc2);
              mv_split(full + (4 + mu) * (9 * LT) + i, LT, vb[mu], acc, acc2);
            }
  #pragma unroll
            for (int a = 0; a < 3; ++a) acc[a] = make_float2(acc[a].x - acc2[a].y, acc[a].y + acc2[a].x);
          } else {
  #pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
              mv_x2(L + mu * (NEL * LT) + i, LT, vf[mu], bf[mu], acc);
              mvdag_x2(L + (4 + mu) * (NEL * LT) + i, LT, vb[mu], -bb[mu], acc);
            }
          }
          if (EPI == EPI_CG_K2) {
            // p = r + beta p_old; A p = 4 m^2 p - D_eo t; r -= alpha A p; x_lo += alpha p
  #pragma unroll
            for (int k = 0; k < 3; ++k) {
              c0[k] = __ffma2_rn(bc2(beta), c0[k], c1[k]);
              const float2 ap = __ffma2_rn(bc2(m4), c0[k], make_float2(-acc[k].x, -acc[k].y));
              c1[k] = __ffma2_rn(bc2(-alpha), ap, c1[k]);
              c2[k] = __ffma2_rn(bc2(alpha), c0[k], c2[k]);
              q0 += c1[k].x * c1[k].x + c1[k].y * c1[k].y;
              q1 += c1[k].x * c0[k].x + c1[k].y * c0[k].y;
            }
            st3(a.center, j, s, Ve, c0);
            st3(a.aux, j, s, Ve, c1);
            st3(a.xlo, j, s, Ve, c2);
          } else {
            // t = D_oe r + beta t_old
  #pragma unroll
            for (int k = 0; k < 3; ++k) {
              c0[k] = __ffma2_rn(bc2(beta), c0[k], acc[k]);
              q0 += c0[k].x * c0[k].x + c0[k].y * c0[k].y;
            }
            st3(a.out, j, s, Ve, c0);
          }
        }
        q0 = warp_sum(q0);
        if (NV > 1) q1 = warp_sum(q1);
        if ((tid & 31) == 0 && has) {
          red[j][warp][0] += q0;
          if (NV > 1) red[j][warp][NV - 1] += q1;
        }
      }
    }
  }
  __syncthreads();
  if (failed) {
    // the copies still outstanding land before the block exits (bounded)
    if (tid == 0)
      for (int q = issued - STG > 0 ? issued - STG : 0; q < issued; ++q) mbar_wait(&bar[q % STG], (unsigned)(q / STG) & 1u);
    __syncthreads();
  }
  // one FP64 partial per system and value: the warps in order
  if (a.ctl.st != nullptr) {
    for (int k = tid; k < nsys * NV; k += BT) {
      const int j = k / NV, v = k % NV;
      float sum = 0.f;
#pragma unroll
      for (int w = 0; w < NW; ++w) sum += red[j][w][v];
      a.ctl.partials[((long long)j * NVMAX + v) * a.ctl.pstride + blockIdx.x] = (double)sum;
    }
  }
}

template <int RC_, int EPI_, int SL_, int STG_, int JJ_>
static cudaError_t nrhs_one(int nblocks, cudaStream_t st, const DsArgs &a, const void **kptr) {
  auto k = k_cg_nrhs<RC_, EPI_, SL_, STG_, JJ_>;
  const unsigned smem = nrhs_smem_bytes(RC_, STG_);
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

// The form each kernel of a mixed form runs.  Form 24: two systems per pass
// in kernel 1 only -- kernel 2 (three more vectors per system in its
// epilogue) measured slower that way and keeps one system per pass (form 4).
int nrhs_kernel_form(int form, int EPI) { return (EPI == EPI_CG_K2 && form == 24) ? 4 : form; }

cudaError_t launch_cg_nrhs(int recon, int form, int EPI, int nblocks, cudaStream_t st, const DsArgs &a,
                           const void **kptr) {
  form = nrhs_kernel_form(form, EPI);
#define STAG_NR(RC_, EPI_, SL_, STG_, JJ_)                                          \
  if (recon == RC_ && EPI == EPI_ && form == 10 * (2 - STG_) + 20 * (JJ_ - 1) + SL_) \
    return nrhs_one<RC_, EPI_, SL_, STG_, JJ_>(nblocks, st, a, kptr);
  STAG_NR(0, EPI_CG_K1R, 2, 2, 1) STAG_NR(0, EPI_CG_K2, 2, 2, 1) STAG_NR(1, EPI_CG_K1R, 2, 2, 1)
  STAG_NR(1, EPI_CG_K2, 2, 2, 1) STAG_NR(0, EPI_CG_K1R, 4, 2, 1) STAG_NR(0, EPI_CG_K2, 4, 2, 1)
  STAG_NR(1, EPI_CG_K1R, 4, 2, 1) STAG_NR(1, EPI_CG_K2, 4, 2, 1) STAG_NR(1, EPI_CG_K1R, 4, 1, 1)
  STAG_NR(1, EPI_CG_K2, 4, 1, 1) STAG_NR(0, EPI_CG_K1R, 4, 1, 1) STAG_NR(0, EPI_CG_K2, 4, 1, 1)
  STAG_NR(1, EPI_CG_K1R, 4, 2, 2)
#undef STAG_NR
  return cudaErrorNotSupported;
}

unsigned cg_nrhs_smem(int recon, int form) { return nrhs_smem_bytes(recon, form == 14 ? 1 : 2); }

}  // namespace stag
