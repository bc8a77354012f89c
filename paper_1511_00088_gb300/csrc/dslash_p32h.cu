// FP32 link-storage instantiations of the half operator with FP16 Krylov
// vectors and a per-site scale (STAG_VEC_FP16): link and vector storage
// chosen independently.
#include "dslash_inst.cuh"
namespace stag {
cudaError_t launch_dslash_p32h(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                               cudaStream_t st, const DsArgs &a, const void **kptr) {
  STAG_DS_EPIS(P32, 0, P16, P16, 1)
  STAG_DS_EPIS(P32, 0, P16, P16, 4)
  STAG_DS_EPIS(P32, 0, P16, P16, 8)
  STAG_DS_EPIS(P32, 1, P16, P16, 1)
  STAG_DS_EPIS(P32, 1, P16, P16, 4)
  STAG_DS_EPIS(P32, 1, P16, P16, 8)
  return cudaErrorNotSupported;
}
}  // namespace stag
