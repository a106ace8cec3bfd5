// Instantiation body shared by the k_m<M>.cu units: defines the lookup
// functions for one template capacity MV and the chunk splits SPL it supports.
#pragma once
#include "mdhp_dispatch.h"

#define MDHP_LLG_CASE(MV, S)                                                             \
  if (SPL == S) {                                                                        \
    if (BM == 0 && !learn) return stage ? k_loglik_grad<MV, S, 0, false, true> : k_loglik_grad<MV, S, 0, false, false>; \
    if (BM == 0 && learn) return stage ? k_loglik_grad<MV, S, 0, true, true> : k_loglik_grad<MV, S, 0, true, false>;    \
    if (BM == 1 && !learn) return stage ? k_loglik_grad<MV, S, 1, false, true> : k_loglik_grad<MV, S, 1, false, false>; \
    if (BM == 1 && learn) return stage ? k_loglik_grad<MV, S, 1, true, true> : k_loglik_grad<MV, S, 1, true, false>;    \
  }

#define MDHP_FIT_CASE(MV, S)                                                             \
  if (SPL == S) {                                                                        \
    if (BM == 0 && !learn) return stage ? k_fit<MV, S, 0, false, true> : k_fit<MV, S, 0, false, false>; \
    if (BM == 0 && learn) return stage ? k_fit<MV, S, 0, true, true> : k_fit<MV, S, 0, true, false>;    \
    if (BM == 1 && !learn) return stage ? k_fit<MV, S, 1, false, true> : k_fit<MV, S, 1, false, false>; \
    if (BM == 1 && learn) return stage ? k_fit<MV, S, 1, true, true> : k_fit<MV, S, 1, true, false>;    \
  }
