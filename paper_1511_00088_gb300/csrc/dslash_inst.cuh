// dslash_inst.cuh -- instantiation table of the half-operator kernel (one
// translation unit per link precision, so they compile in parallel).
#pragma once
#include "launch.h"

namespace stag {
// one instantiation of the half operator: launch it, or (kptr) return it; with
// a.tma = 1 or 2 the tiled-links variant where it exists
template <int LP_, int RC_, int VP_, int OP_, int NS_, int EPI_, int L_>
cudaError_t ds_one(int nblocks, cudaStream_t st, const DsArgs &a, const void **kptr) {
  constexpr bool CAN_TMA =
      NS_ == 1 && LP_ != P64 && (EPI_ == EPI_CG_K1 || EPI_ == EPI_CG_K1R || EPI_ == EPI_CG_K2);
  if constexpr (CAN_TMA) {
    if (a.tma == 2) {
      auto k = k_dslash<LP_, RC_, VP_, OP_, NS_, EPI_, DS_BT, L_, 2>;
      if (kptr) {
        *kptr = (const void *)k;
        return cudaSuccess;
      }
      return launch_ex_full(k, nblocks, DS_BT, 0u, st, a.pdl != 0, a.l2_base, a.l2_bytes, a.l2_hit, a);
    }
    if (a.tma == 1) {
      auto k = k_dslash<LP_, RC_, VP_, OP_, NS_, EPI_, DS_BT, L_, 1>;
      const unsigned smem = tma_smem_bytes(LP_, RC_, L_);
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
      return launch_ex_full(k, nblocks, DS_BT, smem, st, a.pdl != 0, a.l2_base, a.l2_bytes, a.l2_hit, a);
    }
  }
  auto k = k_dslash<LP_, RC_, VP_, OP_, NS_, EPI_, DS_BT, L_>;
  if (kptr) {
    *kptr = (const void *)k;
    return cudaSuccess;
  }
  return launch_ex_full(k, nblocks, DS_BT, 0u, st, a.pdl != 0, a.l2_base, a.l2_bytes, a.l2_hit, a);
}
}  // namespace stag

#define STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_)                                      \
  if (recon == RC_ && VP == VP_ && OP == OP_ && NS == NS_ && EPI == EPI_) {              \
    if (lanes == 2) return ds_one<LP_, RC_, VP_, OP_, NS_, EPI_, 2>(nblocks, st, a, kptr); \
    return ds_one<LP_, RC_, VP_, OP_, NS_, EPI_, 1>(nblocks, st, a, kptr);              \
  }

// operator calls (plain, mass epilogue) and the two kernels of a CG iteration
#define STAG_DS_EPIS(LP_, RC_, VP_, OP_, NS_)                \
  STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_PLAIN)          \
  STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_MDAGM)          \
  STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_CG_K1)          \
  STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_CG_K1R)         \
  STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_CG_K2)
