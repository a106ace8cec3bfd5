// Kernel instantiations for template capacity M = 4.
#include "k_inst.cuh"

namespace mdhp {

LlgFn get_llg_m4(int SPL, int BM, bool learn, bool stage) {
  MDHP_LLG_CASE(4, 1)
  return nullptr;
}

FitFn get_fit_m4(int SPL, int BM, bool learn, bool stage) {
  MDHP_FIT_CASE(4, 1)
  return nullptr;
}

WgFn get_wg_m4(int BM) { return BM == 0 ? k_weight_grad<4, 0> : k_weight_grad<4, 1>; }

FitFn get_fitx_m4(int BM, bool xs) {
  if (BM == 0) return xs ? k_fit_x<4, 0, true> : k_fit_x<4, 0, false>;
  return xs ? k_fit_x<4, 1, true> : k_fit_x<4, 1, false>;
}

}  // namespace mdhp
