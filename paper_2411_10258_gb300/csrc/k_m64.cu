// Kernel instantiations for template capacity M = 64.
#include "k_inst.cuh"

namespace mdhp {

LlgFn get_llg_m64(int SPL, int BM, bool learn, bool stage) {
  MDHP_LLG_CASE(64, 8)
  MDHP_LLG_CASE(64, 16)
  return nullptr;
}

FitFn get_fit_m64(int SPL, int BM, bool learn, bool stage) {
  MDHP_FIT_CASE(64, 8)
  MDHP_FIT_CASE(64, 16)
  return nullptr;
}

WgFn get_wg_m64(int BM) { return BM == 0 ? k_weight_grad<64, 0> : k_weight_grad<64, 1>; }

FitFn get_fitx_m64(int, int, int) { return nullptr; }

}  // namespace mdhp
