// Kernel instantiations for template capacity M = 16.
#include "k_inst.cuh"

namespace mdhp {

LlgFn get_llg_m16(int SPL, int BM, bool learn, bool stage) {
  MDHP_LLG_CASE(16, 2)
  MDHP_LLG_CASE(16, 4)
  return nullptr;
}

FitFn get_fit_m16(int SPL, int BM, bool learn, bool stage) {
  MDHP_FIT_CASE(16, 2)
  MDHP_FIT_CASE(16, 4)
  return nullptr;
}

WgFn get_wg_m16(int BM) { return BM == 0 ? k_weight_grad<16, 0> : k_weight_grad<16, 1>; }

FitFn get_fitx_m16(int BM, int xm, int nt) {
  if (BM == 2) {  // matrix beta (fixed): global or shared-memory features
    if (xm == XM_SHARED) return k_fit_x<16, 2, XM_SHARED, 0>;
    if (xm != XM_GLOBAL) return nullptr;
    switch (nt) {
      case 64: return k_fit_x<16, 2, XM_GLOBAL, 64>;
      case 128: return k_fit_x<16, 2, XM_GLOBAL, 128>;
      case 256: return k_fit_x<16, 2, XM_GLOBAL, 256>;
    }
    return nullptr;
  }
  if (BM != 0 && BM != 1) return nullptr;
  if (xm == XM_SHARED) return BM == 0 ? k_fit_x<16, 0, XM_SHARED, 0> : k_fit_x<16, 1, XM_SHARED, 0>;
  if (xm == XM_RING) return BM == 0 ? k_fit_x<16, 0, XM_RING, 0> : k_fit_x<16, 1, XM_RING, 0>;
  if (xm != XM_GLOBAL) return nullptr;
  switch (nt) {  // block size compiled in: constant-offset feature loads
    case 64: return BM == 0 ? k_fit_x<16, 0, XM_GLOBAL, 64> : k_fit_x<16, 1, XM_GLOBAL, 64>;
    case 128: return BM == 0 ? k_fit_x<16, 0, XM_GLOBAL, 128> : k_fit_x<16, 1, XM_GLOBAL, 128>;
    case 256: return BM == 0 ? k_fit_x<16, 0, XM_GLOBAL, 256> : k_fit_x<16, 1, XM_GLOBAL, 256>;
  }
  return nullptr;
}

}  // namespace mdhp
