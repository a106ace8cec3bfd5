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

}  // namespace mdhp
