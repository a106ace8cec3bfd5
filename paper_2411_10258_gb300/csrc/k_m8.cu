// Kernel instantiations for template capacity M = 8.
#include "k_inst.cuh"

namespace mdhp {

LlgFn get_llg_m8(int SPL, int BM, bool learn, bool stage) {
  MDHP_LLG_CASE(8, 2)
  return nullptr;
}

FitFn get_fit_m8(int SPL, int BM, bool learn, bool stage) {
  MDHP_FIT_CASE(8, 2)
  return nullptr;
}

WgFn get_wg_m8(int BM) { return BM == 0 ? k_weight_grad<8, 0> : k_weight_grad<8, 1>; }

FitFn get_fitx_m8(int BM, int xm, int nt) {
  if (BM == 2) {  // matrix beta (fixed): global or shared-memory features
    if (xm == XM_SHARED) return k_fit_x<8, 2, XM_SHARED, 0>;
    if (xm != XM_GLOBAL) return nullptr;
    switch (nt) {
      case 64: return k_fit_x<8, 2, XM_GLOBAL, 64>;
      case 128: return k_fit_x<8, 2, XM_GLOBAL, 128>;
      case 256: return k_fit_x<8, 2, XM_GLOBAL, 256>;
    }
    return nullptr;
  }
  if (BM != 0 && BM != 1) return nullptr;
  if (xm == XM_SHARED) return BM == 0 ? k_fit_x<8, 0, XM_SHARED, 0> : k_fit_x<8, 1, XM_SHARED, 0>;
  if (xm == XM_RING) return BM == 0 ? k_fit_x<8, 0, XM_RING, 0> : k_fit_x<8, 1, XM_RING, 0>;
  if (xm != XM_GLOBAL) return nullptr;
  switch (nt) {  // block size compiled in: constant-offset feature loads
    case 64: return BM == 0 ? k_fit_x<8, 0, XM_GLOBAL, 64> : k_fit_x<8, 1, XM_GLOBAL, 64>;
    case 128: return BM == 0 ? k_fit_x<8, 0, XM_GLOBAL, 128> : k_fit_x<8, 1, XM_GLOBAL, 128>;
    case 256: return BM == 0 ? k_fit_x<8, 0, XM_GLOBAL, 256> : k_fit_x<8, 1, XM_GLOBAL, 256>;
  }
  return nullptr;
}

}  // namespace mdhp
