// Instantiations of the shared-memory multi-system CG kernels (FP32 links and
// vectors, 4 or 8 systems per block).
#include "launch.h"

namespace stag {

template <int RC_, int NSW_, int EPI_>
static cudaError_t mrhs_one(int nblocks, cudaStream_t st, const DsArgs &a, const void **kptr) {
  auto k = k_dslash_mrhs<P32, RC_, NSW_, EPI_>;
  if (kptr) {
    *kptr = (const void *)k;
    return cudaSuccess;
  }
  return launch_ex_full(k, nblocks, 32 * NSW_, 0u, st, a.pdl != 0, a.l2_base, a.l2_bytes, a.l2_hit, a);
}

cudaError_t launch_dslash_mrhs(int LP, int recon, int nsw, int EPI, int nblocks, cudaStream_t st, const DsArgs &a,
                               const void **kptr) {
  if (LP != P32) return cudaErrorNotSupported;
#define STAG_MR(RC_, NSW_, EPI_)                                                \
  if (recon == RC_ && nsw == NSW_ && EPI == EPI_) return mrhs_one<RC_, NSW_, EPI_>(nblocks, st, a, kptr);
  STAG_MR(0, 4, EPI_CG_K1R) STAG_MR(0, 4, EPI_CG_K2) STAG_MR(0, 8, EPI_CG_K1R) STAG_MR(0, 8, EPI_CG_K2)
  STAG_MR(1, 4, EPI_CG_K1R) STAG_MR(1, 4, EPI_CG_K2) STAG_MR(1, 8, EPI_CG_K1R) STAG_MR(1, 8, EPI_CG_K2)
#undef STAG_MR
  return cudaErrorNotSupported;
}

}  // namespace stag
