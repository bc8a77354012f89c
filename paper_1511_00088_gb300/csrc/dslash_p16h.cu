// P16 link-storage instantiations of the half operator with P16 Krylov
// vectors and a per-site scale (STAG_HALF_VECTORS, STAG_ROUND_OUTPUT).
#include "dslash_inst.cuh"
namespace stag {
cudaError_t launch_dslash_p16h(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                               cudaStream_t st, const DsArgs &a, const void **kptr) {
  STAG_DS_EPIS(P16, 0, P16, P16, 1)
  STAG_DS_EPIS(P16, 0, P16, P16, 4)
  STAG_DS_EPIS(P16, 0, P16, P16, 8)
  STAG_DS_EPIS(P16, 1, P16, P16, 1)
  STAG_DS_EPIS(P16, 1, P16, P16, 4)
  STAG_DS_EPIS(P16, 1, P16, P16, 8)
  return cudaErrorNotSupported;
}
}  // namespace stag
