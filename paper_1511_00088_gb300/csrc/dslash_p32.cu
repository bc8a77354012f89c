// FP32 instantiations of the half operator (full and reconstruct-12 links)
// with FP32 Krylov vectors; those with FP16 / BF16 vectors are in
// dslash_p32h.cu / dslash_p32b.cu, compiled in parallel.
#include "dslash_inst.cuh"
namespace stag {
cudaError_t launch_dslash_p32h(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                               cudaStream_t st, const DsArgs &a, const void **kptr);
cudaError_t launch_dslash_p32b(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                               cudaStream_t st, const DsArgs &a, const void **kptr);

cudaError_t launch_dslash_p32(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                              cudaStream_t st, const DsArgs &a, const void **kptr) {
  STAG_DS_EPIS(P32, 0, P32, P32, 1)
  STAG_DS_EPIS(P32, 0, P32, P32, 4)
  STAG_DS_EPIS(P32, 0, P32, P32, 8)
  STAG_DS_EPIS(P32, 1, P32, P32, 1)
  STAG_DS_EPIS(P32, 1, P32, P32, 4)
  STAG_DS_EPIS(P32, 1, P32, P32, 8)
  if (VP == P16) return launch_dslash_p32h(recon, VP, OP, NS, EPI, lanes, nblocks, st, a, kptr);
  if (VP == PBF) return launch_dslash_p32b(recon, VP, OP, NS, EPI, lanes, nblocks, st, a, kptr);
  return cudaErrorNotSupported;
}
}  // namespace stag
