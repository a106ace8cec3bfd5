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

FitFn get_fitx_m32(int BM, bool xs) {
  if (BM == 0) return xs ? k_fit_x<32, 0, true> : k_fit_x<32, 0, false>;
  return xs ? k_fit_x<32, 1, true> : k_fit_x<32, 1, false>;
}

}  // namespace mdhp
