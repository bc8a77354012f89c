// dslash_inst.cuh -- instantiation table of the half-operator kernel (one
// translation unit per link precision, so they compile in parallel).
#pragma once
#include "launch.h"

#define STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_)                                      \
  if (recon == RC_ && VP == VP_ && OP == OP_ && NS == NS_ && EPI == EPI_) {              \
    if (kptr != nullptr) {                                                               \
      *kptr = (lanes == 2) ? (const void *)k_dslash<LP_, RC_, VP_, OP_, NS_, EPI_, DS_BT, 2> \
                           : (const void *)k_dslash<LP_, RC_, VP_, OP_, NS_, EPI_, DS_BT, 1>; \
      return cudaSuccess;                                                                \
    }                                                                                    \
    if (lanes == 2)                                                                      \
      return launch_ex(k_dslash<LP_, RC_, VP_, OP_, NS_, EPI_, DS_BT, 2>, nblocks, DS_BT, st, \
                       a.pdl != 0, a);                                                   \
    return launch_ex(k_dslash<LP_, RC_, VP_, OP_, NS_, EPI_, DS_BT, 1>, nblocks, DS_BT, st,   \
                     a.pdl != 0, a);                                                     \
  }

// operator calls (plain, mass epilogue) and the two kernels of a CG iteration
#define STAG_DS_EPIS(LP_, RC_, VP_, OP_, NS_)                \
  STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_PLAIN)          \
  STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_MDAGM)          \
  STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_CG_K1)          \
  STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_CG_K1R)         \
  STAG_DS_CASE(LP_, RC_, VP_, OP_, NS_, EPI_CG_K2)
