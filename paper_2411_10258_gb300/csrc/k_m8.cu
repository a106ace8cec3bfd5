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

FitFn get_fitx_m8(int BM, bool xs) {
  if (BM == 0) return xs ? k_fit_x<8, 0, true> : k_fit_x<8, 0, false>;
  return xs ? k_fit_x<8, 1, true> : k_fit_x<8, 1, false>;
}

}  // namespace mdhp
