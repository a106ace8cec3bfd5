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

FitFn get_fitx_m16(int BM, bool xs) {
  if (BM == 0) return xs ? k_fit_x<16, 0, true> : k_fit_x<16, 0, false>;
  return xs ? k_fit_x<16, 1, true> : k_fit_x<16, 1, false>;
}

}  // namespace mdhp
