// Host-only C entry points: status strings and the exact planner queries.
#include <cstring>
#include <vector>

#include "../../include/pfft.h"
#include "lattice.hpp"

using namespace pfft;

extern "C" const char* pfft_status_string(pfft_status s) {
  switch (s) {
    case PFFT_OK: return "ok";
    case PFFT_ERR_ARG: return "invalid argument";
    case PFFT_ERR_SINGULAR: return "singular matrix";
    case PFFT_ERR_OVERFLOW: return "size or entry beyond the supported range";
    case PFFT_ERR_NOT_INTEGRAL: return "J^{-1} M is not an integer matrix";
    case PFFT_ERR_UNSUPPORTED: return "unsupported shape for the transform kernels";
    case PFFT_ERR_OOM: return "device allocation failed";
    case PFFT_ERR_CUDA: return "CUDA runtime error";
    case PFFT_ERR_TIMEOUT: return "device wait timed out";
    case PFFT_ERR_DEVICE_CHECK: return "device-side check failed";
  }
  return "unknown status";
}

static pfft_status load(int d, const int64_t* M, IMat& A) {
  if (d < 1 || d > 4 || !M) return PFFT_ERR_ARG;
  A = IMat(d);
  for (int i = 0; i < d * d; ++i) {
    if (M[i] >= (int64_t(1) << 24) || M[i] <= -(int64_t(1) << 24)) return PFFT_ERR_OVERFLOW;
    A.a[i] = M[i];
  }
  try {
    if (determinant(A) == 0) return PFFT_ERR_SINGULAR;
  } catch (const LatticeError& e) {
    return pfft_status(e.code);
  }
  return PFFT_OK;
}

extern "C" pfft_status pfft_hermite_normal_form(int d, const int64_t* M, int64_t* H) {
  if (!H) return PFFT_ERR_ARG;
  IMat A;
  pfft_status st = load(d, M, A);
  if (st != PFFT_OK) return st;
  try {
    IMat R = hermite_normal_form(A);
    std::memcpy(H, R.a.data(), sizeof(int64_t) * d * d);
  } catch (const LatticeError& e) {
    return pfft_status(e.code);
  }
  return PFFT_OK;
}

extern "C" pfft_status pfft_smith_normal_form(int d, const int64_t* M, int64_t* Q, int64_t* eps,
                                              int64_t* R) {
  if (!Q || !eps || !R) return PFFT_ERR_ARG;
  IMat A;
  pfft_status st = load(d, M, A);
  if (st != PFFT_OK) return st;
  try {
    IMat Qm, Rm, U, V;
    std::vector<i64> e;
    smith_normal_form(A, Qm, e, Rm, U, V);
    std::memcpy(Q, Qm.a.data(), sizeof(int64_t) * d * d);
    std::memcpy(R, Rm.a.data(), sizeof(int64_t) * d * d);
    std::memcpy(eps, e.data(), sizeof(int64_t) * d);
  } catch (const LatticeError& e) {
    return pfft_status(e.code);
  }
  return PFFT_OK;
}
