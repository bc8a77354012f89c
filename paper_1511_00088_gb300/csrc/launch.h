// launch.h -- host-side launchers of libstag's kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "stag_kernels.cuh"

namespace stag {

constexpr int DS_BT = 128;    // threads per block of the half-operator kernels

// blocks of the half operator for Ve sites with `lanes` lanes per site
inline int ds_blocks(int Ve, int lanes) {
  const int sites = DS_BT / lanes;
  return (Ve + sites - 1) / sites;
}
constexpr int BLAS_BT = 256;  // threads per block of the BLAS-1 kernels

// Launch kernel k on nblocks x bt threads in stream st.  With pdl the launch
// carries programmatic stream serialisation: k may be scheduled while the
// previous kernel in the stream drains, and must reach grid_dep_wait() before
// it reads or writes anything that kernel touches.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_ex_full(void (*k)(KArgs...), int nblocks, int bt, unsigned smem, cudaStream_t st,
                                  bool pdl, const void *l2_base, size_t l2_bytes, float l2_hit, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nblocks);
  cfg.blockDim = dim3((unsigned)bt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  unsigned n = 0;
  if (pdl) {
    at[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
  }
  if (l2_bytes > 0) {
    // a fraction l2_hit of the window's lines persists in L2 across kernels
    at[n].id = cudaLaunchAttributeAccessPolicyWindow;
    at[n].val.accessPolicyWindow.base_ptr = const_cast<void *>(l2_base);
    at[n].val.accessPolicyWindow.num_bytes = l2_bytes;
    at[n].val.accessPolicyWindow.hitRatio = l2_hit;
    at[n].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    at[n].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    ++n;
  }
  cfg.attrs = at;
  cfg.numAttrs = n;
  return cudaLaunchKernelEx(&cfg, k, static_cast<Args &&>(args)...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_ex_smem(void (*k)(KArgs...), int nblocks, int bt, unsigned smem, cudaStream_t st,
                                  bool pdl, Args &&...args) {
  return launch_ex_full(k, nblocks, bt, smem, st, pdl, nullptr, 0, 0.f, static_cast<Args &&>(args)...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_ex(void (*k)(KArgs...), int nblocks, int bt, cudaStream_t st, bool pdl,
                             Args &&...args) {
  return launch_ex_smem(k, nblocks, bt, 0u, st, pdl, static_cast<Args &&>(args)...);
}

// dynamic shared memory of a half-operator kernel with bulk-copied links
// (DsArgs::tma): TMA_STAGES chunks of DS_BT / lanes sites x 8 links
inline unsigned tma_smem_bytes(int LP, int recon, int lanes) {
  const unsigned cb = (LP == P32) ? 8u : 4u;
  return (unsigned)TMA_STAGES * (unsigned)(DS_BT / lanes) * 8u * (recon ? 6u : 9u) * cb;
}
// tiles per parity of the tiled site-owned links (whole chunks of DS_BT sites)
inline int link_tiles(int Ve) { return (Ve + DS_BT - 1) / DS_BT * (DS_BT / LT); }

// Launch k_dslash<LP, recon, VP, OP, NS, EPI, DS_BT, lanes> on `nblocks`
// blocks (lanes = 1 or 2 lanes per output site).  Returns
// cudaErrorNotSupported for a combination the library does not instantiate.
// With kptr != nullptr nothing is launched: *kptr receives the kernel (for
// occupancy queries).
cudaError_t launch_dslash(int LP, int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                          cudaStream_t st, const DsArgs &a, const void **kptr = nullptr);
cudaError_t launch_dslash_p64(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                              cudaStream_t st, const DsArgs &a, const void **kptr);
cudaError_t launch_dslash_p32(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                              cudaStream_t st, const DsArgs &a, const void **kptr);
cudaError_t launch_dslash_p16(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                              cudaStream_t st, const DsArgs &a, const void **kptr);
cudaError_t launch_dslash_pbf(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                              cudaStream_t st, const DsArgs &a, const void **kptr);

// k_dslash_mrhs<LP, recon, nsw, EPI> (LP = P32; nsw = 4 or 8 systems per block
// of 32 nsw threads; EPI_CG_K1R or EPI_CG_K2) on nblocks blocks; kptr as above
cudaError_t launch_dslash_mrhs(int LP, int recon, int nsw, int EPI, int nblocks, cudaStream_t st, const DsArgs &a,
                               const void **kptr = nullptr);

// k_cg_nrhs (nrhs.cu): the two CG kernels for nsys <= 64 systems, FP32
// links (tiled copy, a.links_tile) and vectors; form = sl (2 or 4 threads per
// site, two link stages) or 10 + sl (one stage, 3 blocks per SM; sl = 4);
// nblocks blocks stride over tiles of LT sites; kptr as above
cudaError_t launch_cg_nrhs(int recon, int form, int EPI, int nblocks, cudaStream_t st, const DsArgs &a,
                           const void **kptr = nullptr);
unsigned cg_nrhs_smem(int recon, int form);
int nrhs_kernel_form(int form, int EPI);
constexpr int CG_NRHS_MAX = 64;

cudaError_t launch_accum_x(int RP, int NS, int nblocks, cudaStream_t st, const BlasArgs &a);
// multi-shift CG (multishift.cu): the shifted-system update between the two CG
// kernels (a.nbx blocks per base system), and the pending-update mark of a
// solve from an initial guess
cudaError_t launch_shift_update(const MsArgs &a, cudaStream_t st);
cudaError_t launch_mark_update(SysState *st, int nsys, cudaStream_t s);
// k_finalize over the partials of the kernel just launched: nbx blocks per
// system group, nv values per system (pdl: launched as a programmatic
// dependent of that kernel)
cudaError_t launch_finalize(const Ctl &c, int fin, int nbx, int nv, int nsys, cudaStream_t st,
                            bool pdl = false, const SysState *st_in = nullptr);
cudaError_t launch_cg_init(int VP, int RP, int NS, int nblocks, cudaStream_t st, const BlasArgs &a);

cudaError_t launch_pack_vec(int P, const double2 *src, VecArg dst, int k, int Ve, cudaStream_t st);
// full-lattice ABI vector [V][3] -> system k of the even / odd halves (FP64), and back
cudaError_t launch_split_full(const double2 *full, VecArg e, VecArg o, int k, Geom g, cudaStream_t st);
cudaError_t launch_merge_full(VecArg e, int ke, VecArg o, int ko, double2 *full, Geom g, cudaStream_t st);
cudaError_t launch_unpack_vec(int P, VecArg src, int k, double2 *dst, int Ve, cudaStream_t st);
cudaError_t launch_convert_vec(int PIN, int POUT, VecArg src, VecArg dst, int nsys, int Ve,
                               cudaStream_t st);
cudaError_t launch_pack_links(int LP, int recon, const double2 *src, void *dst, Geom g,
                              cudaStream_t st);
// the tiled site-owned copy (LP = P32, P16 or PBF); dst already zeroed
cudaError_t launch_pack_links_tiled(int LP, int recon, const double2 *src, void *dst, Geom g, int ntile,
                                    cudaStream_t st);
cudaError_t launch_su3_defect(const double2 *U, long long nlinks, unsigned long long *out,
                              cudaStream_t st);

// NPR one-colour-trace four-fermion contraction (npr.cu): out[h] = O(z_h) for
// every hypercube (V / 16 entries), *sum (may be null) = their sum; U the
// canonical [4][V][3][3] links, fields [V][3]; st = (S1, F1, S2, F2), 4-bit corner masks
cudaError_t launch_npr(const int dims[4], const double2 *U, const int st[4], const double2 *cb1, const double2 *c2,
                       const double2 *cb3, const double2 *c4, double2 *out, double2 *sum, cudaStream_t s);

// HYP smearing (hyp.cu): out [4][V][3][3] = the smeared links of U (same
// layout; out may alias U); Vb, Vt scratch of 12 V links each; alpha = (a1, a2, a3)
cudaError_t launch_hyp(const int dims[4], const double2 *U, const double alpha[3], double2 *Vb, double2 *Vt,
                       double2 *out, cudaStream_t st);

// k_force over all 4 V links (force.cu): X even, Y = D_oe X odd (device SoA,
// FP64); grad [4][V][3][3] complex and/or lie [4][V][8] (either may be null)
cudaError_t launch_force(Geom g, const double2 *X, const double2 *Y, const void *links64, double2 *grad,
                         double *lie, double scale, cudaStream_t st);
// S = 2 Re<phi, x> - Re<x, ax> over Ve sites of one system (FP64 SoA), in
// double-word arithmetic and a fixed order: part holds 2 action_blocks(Ve)
// doubles of scratch, *out (device) receives S
int action_blocks(int Ve);
cudaError_t launch_action(VecArg phi, VecArg x, VecArg ax, int Ve, double *part, double *out, cudaStream_t st);
// out[i] = a x[i], i < n (FP64)
cudaError_t launch_scale_reals(const double *x, double a, double *out, long long n, cudaStream_t st);

}  // namespace stag
