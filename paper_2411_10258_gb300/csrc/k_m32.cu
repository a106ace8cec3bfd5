// Kernel instantiations for template capacity M = 32.
#include "k_inst.cuh"

namespace mdhp {

LlgFn get_llg_m32(int SPL, int BM, bool learn, bool stage) {
  MDHP_LLG_CASE(32, 4)
  MDHP_LLG_CASE(32, 8)
  return nullptr;
}

FitFn get_fit_m32(int SPL, int BM, bool learn, bool stage) {
  MDHP_FIT_CASE(32, 4)
  MDHP_FIT_CASE(32, 8)
  return nullptr;
}

WgFn get_wg_m32(int BM) { return BM == 0 ? k_weight_grad<32, 0> : k_weight_grad<32, 1>; }

FitFn get_fitx_m32(int BM, int xm, int nt) {
  if (BM == 2) {  // matrix beta (fixed): global or shared-memory features
    if (xm == XM_SHARED) return k_fit_x<32, 2, XM_SHARED, 0>;
    if (xm != XM_GLOBAL) return nullptr;
    switch (nt) {
      case 64: return k_fit_x<32, 2, XM_GLOBAL, 64>;
      case 128: return k_fit_x<32, 2, XM_GLOBAL, 128>;
      case 256: return k_fit_x<32, 2, XM_GLOBAL, 256>;
    }
    return nullptr;
  }
  if (BM != 0 && BM != 1) return nullptr;
  if (xm == XM_SHARED) return BM == 0 ? k_fit_x<32, 0, XM_SHARED, 0> : k_fit_x<32, 1, XM_SHARED, 0>;
  if (xm == XM_RING) return BM == 0 ? k_fit_x<32, 0, XM_RING, 0> : k_fit_x<32, 1, XM_RING, 0>;
  if (xm == XM_TMEM) {  // tensor-memory feature rows: 256 threads, one CTA per SM
    if (nt == 256) return BM == 0 ? k_fit_x<32, 0, XM_TMEM, 256> : k_fit_x<32, 1, XM_TMEM, 256>;
    if (nt == 384) return BM == 0 ? k_fit_x<32, 0, XM_TMEM, 384> : k_fit_x<32, 1, XM_TMEM, 384>;
    return nullptr;  // 128 threads at two CTAs per SM measured slower than the scratch alone
  }
  if (xm != XM_GLOBAL) return nullptr;
  switch (nt) {  // block size compiled in: constant-offset feature loads
    case 64: return BM == 0 ? k_fit_x<32, 0, XM_GLOBAL, 64> : k_fit_x<32, 1, XM_GLOBAL, 64>;
    case 128: return BM == 0 ? k_fit_x<32, 0, XM_GLOBAL, 128> : k_fit_x<32, 1, XM_GLOBAL, 128>;
    case 256: return BM == 0 ? k_fit_x<32, 0, XM_GLOBAL, 256> : k_fit_x<32, 1, XM_GLOBAL, 256>;
  }
  return nullptr;
}

}  // namespace mdhp
