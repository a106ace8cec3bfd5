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
// decoupled fit: xm = XM_GLOBAL (features streamed, register prefetch; built
// for block sizes nt = 64, 128, 256), XM_SHARED (features in shared memory)
// or XM_RING (streamed through a bulk-copy ring); nt is ignored for the last two
FitFn get_fitx(int M, int BM, int xm, int nt);
void record_error(const char *msg);

// Default launch shape of the event-recursion kernels per template capacity
// Mt: threads per window, threads per chunk (sources split across spl
// threads), and the longest window staged in shared memory (mdhp_api.cu).
struct Shape {
  int nt, spl, cutoff;
};
Shape default_shape(int Mt);

#define MDHP_DECLARE_M(MV)                                                   \
  LlgFn get_llg_m##MV(int SPL, int BM, bool learn, bool stage);              \
  FitFn get_fit_m##MV(int SPL, int BM, bool learn, bool stage);              \
  WgFn get_wg_m##MV(int BM);                                                 \
  FitFn get_fitx_m##MV(int BM, int xm, int nt);
MDHP_DECLARE_M(4)
MDHP_DECLARE_M(8)
MDHP_DECLARE_M(16)
MDHP_DECLARE_M(32)
MDHP_DECLARE_M(64)
#undef MDHP_DECLARE_M

}  // namespace mdhp
