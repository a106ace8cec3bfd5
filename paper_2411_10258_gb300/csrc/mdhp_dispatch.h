// Internal: kernel lookup by compile-time shape.  Each template dimension
// capacity M in {4, 8, 16, 32, 64} is instantiated in its own translation unit
// (k_m<M>.cu) so the library compiles in parallel.
#pragma once

#include "mdhp_kernels.cuh"
#include "mdhp_fitx.cuh"

namespace mdhp {

using LlgFn = void (*)(LlgArgs);
using FitFn = void (*)(FitArgs);
using WgFn = void (*)(WgArgs);

// nullptr if the combination is not instantiated
LlgFn get_llg(int M, int SPL, int BM, bool learn, bool stage);
FitFn get_fit(int M, int SPL, int BM, bool learn, bool stage);
WgFn get_wg(int M, int BM);
FitFn get_fitx(int M, int BM, bool xs);
void record_error(const char *msg);

#define MDHP_DECLARE_M(MV)                                                   \
  LlgFn get_llg_m##MV(int SPL, int BM, bool learn, bool stage);              \
  FitFn get_fit_m##MV(int SPL, int BM, bool learn, bool stage);              \
  WgFn get_wg_m##MV(int BM);                                                 \
  FitFn get_fitx_m##MV(int BM, bool xs);
MDHP_DECLARE_M(4)
MDHP_DECLARE_M(8)
MDHP_DECLARE_M(16)
MDHP_DECLARE_M(32)
MDHP_DECLARE_M(64)
#undef MDHP_DECLARE_M

}  // namespace mdhp
