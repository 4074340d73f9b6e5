// Exact integer lattice algebra for the host planner.  See lattice.hpp.
#include "lattice.hpp"

#include <algorithm>
#include <cstdlib>

#include "../../include/pfft.h"

namespace pfft {

static const i128 kLimit = (i128)1 << 100;  // working-value bound before we call it overflow

static i64 narrow(i128 v) {
  if (v > (i128)INT64_MAX || v < (i128)INT64_MIN)
    throw LatticeError{PFFT_ERR_OVERFLOW, "integer overflow in lattice arithmetic"};
  return (i64)v;
}

IMat IMat::identity(int d) {
  IMat I(d);
  for (int i = 0; i < d; ++i) I(i, i) = 1;
  return I;
}

IMat IMat::transpose() const {
  IMat T(d);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) T(i, j) = (*this)(j, i);
  return T;
}

IMat matmul(const IMat& A, const IMat& B) {
  IMat C(A.d);
  for (int i = 0; i < A.d; ++i)
    for (int j = 0; j < A.d; ++j) {
      i128 s = 0;
      for (int k = 0; k < A.d; ++k) s += (i128)A(i, k) * B(k, j);
      C(i, j) = narrow(s);
    }
  return C;
}

i64 gcd64(i64 a, i64 b) {
  a = a < 0 ? -a : a;
  b = b < 0 ? -b : b;
  while (b) {
    i64 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

i64 floordiv(i64 a, i64 b) {
  i64 q = a / b;
  if ((a % b) != 0 && (a < 0)) --q;
  return q;
}

i64 posmod(i64 a, i64 b) {
  i64 r = a % b;
  return r < 0 ? r + b : r;
}

i64 modinv(i64 a, i64 m) {  // extended Euclid
  i64 g0 = posmod(a, m), g1 = m, x0 = 1, x1 = 0;
  while (g1) {
    i64 q = g0 / g1, t;
    t = g0 - q * g1; g0 = g1; g1 = t;
    t = x0 - q * x1; x0 = x1; x1 = t;
  }
  return posmod(x0, m);
}

// Checked i128 steps: an intermediate that leaves the i128 range is an
// overflow error, never a wrapped value.
static i128 mul_checked(i128 a, i128 b) {
  i128 r;
  if (__builtin_mul_overflow(a, b, &r)) throw LatticeError{PFFT_ERR_OVERFLOW, "determinant overflow"};
  return r;
}
static i128 add_checked(i128 a, i128 b) {
  i128 r;
  if (__builtin_add_overflow(a, b, &r)) throw LatticeError{PFFT_ERR_OVERFLOW, "determinant overflow"};
  return r;
}

// Cofactor expansion along the first row.  For d <= 4 and entries below 2^24
// every term is a product of d entries (< 2^96), so the sum is exact; larger
// inputs raise PFFT_ERR_OVERFLOW through the checked steps.
static i128 det_cofactor(const std::vector<i128>& A, int d) {
  if (d == 1) return A[0];
  std::vector<i128> minor(size_t(d - 1) * (d - 1));
  i128 s = 0;
  for (int j = 0; j < d; ++j) {
    if (A[j] == 0) continue;
    for (int r = 1; r < d; ++r)
      for (int c = 0, cc = 0; c < d; ++c)
        if (c != j) minor[size_t(r - 1) * (d - 1) + cc++] = A[size_t(r) * d + c];
    const i128 t = mul_checked(A[j], det_cofactor(minor, d - 1));
    s = add_checked(s, (j & 1) ? -t : t);
  }
  return s;
}

i64 determinant(const IMat& M) {
  const int d = M.d;
  std::vector<i128> A(M.a.begin(), M.a.end());
  if (d <= 4) return narrow(det_cofactor(A, d));
  // fraction-free elimination (Bareiss) for larger d, every product checked
  auto at = [&](int i, int j) -> i128& { return A[size_t(i) * d + j]; };
  i128 prev = 1;
  int sign = 1;
  for (int k = 0; k < d - 1; ++k) {
    if (at(k, k) == 0) {
      int p = -1;
      for (int r = k + 1; r < d; ++r)
        if (at(r, k) != 0) { p = r; break; }
      if (p < 0) return 0;
      for (int j = 0; j < d; ++j) std::swap(at(k, j), at(p, j));
      sign = -sign;
    }
    for (int i = k + 1; i < d; ++i)
      for (int j = k + 1; j < d; ++j) {
        const i128 v = add_checked(mul_checked(at(i, j), at(k, k)), -mul_checked(at(i, k), at(k, j)));
        at(i, j) = v / prev;  // exact division (Bareiss)
        if (at(i, j) > kLimit || at(i, j) < -kLimit)
          throw LatticeError{PFFT_ERR_OVERFLOW, "determinant overflow"};
      }
    prev = at(k, k);
  }
  return narrow(sign * at(d - 1, d - 1));
}

IMat adjugate(const IMat& M) {
  const int d = M.d;
  IMat A(d);
  if (d == 1) {
    A(0, 0) = 1;
    return A;
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      IMat minor(d - 1);
      for (int r = 0, rr = 0; r < d; ++r) {
        if (r == j) continue;
        for (int c = 0, cc = 0; c < d; ++c) {
          if (c == i) continue;
          minor(rr, cc++) = M(r, c);
        }
        ++rr;
      }
      i64 v = determinant(minor);
      A(i, j) = ((i + j) & 1) ? -v : v;
    }
  return A;
}

bool inverse_unimodular(const IMat& U, IMat& inv) {
  i64 D = determinant(U);
  if (D != 1 && D != -1) return false;
  inv = adjugate(U);
  if (D == -1)
    for (auto& x : inv.a) x = -x;
  return true;
}

namespace {
struct BigMat {  // working copy with 128-bit entries and overflow guard
  int d;
  std::vector<i128> a;
  explicit BigMat(const IMat& M) : d(M.d), a(M.a.begin(), M.a.end()) {}
  i128& operator()(int i, int j) { return a[size_t(i) * d + j]; }
  void check() const {
    for (auto v : a)
      if (v > kLimit || v < -kLimit) throw LatticeError{PFFT_ERR_OVERFLOW, "lattice reduction overflow"};
  }
  IMat narrowed() const {
    IMat M(d);
    for (size_t i = 0; i < a.size(); ++i) M.a[i] = narrow(a[i]);
    return M;
  }
};
i128 fdiv128(i128 a, i128 b) {  // floor division
  i128 q = a / b;
  if ((a % b) != 0 && ((a < 0) != (b < 0))) --q;
  return q;
}
i128 abs128(i128 v) { return v < 0 ? -v : v; }
}  // namespace

IMat hermite_normal_form(const IMat& Min) {
  const int d = Min.d;
  BigMat A(Min);
  auto colop = [&](int dst, int src, i128 q) {
    if (q == 0) return;
    for (int i = 0; i < d; ++i) A(i, dst) -= q * A(i, src);
  };
  for (int r = d - 1; r >= 0; --r) {
    for (;;) {
      int piv = -1;
      for (int c = 0; c <= r; ++c)
        if (A(r, c) != 0 && (piv < 0 || abs128(A(r, c)) < abs128(A(r, piv)))) piv = c;
      if (piv < 0) throw LatticeError{PFFT_ERR_SINGULAR, "singular matrix"};
      bool done = true;
      for (int c = 0; c <= r; ++c)
        if (c != piv && A(r, c) != 0) {
          colop(c, piv, fdiv128(A(r, c), A(r, piv)));
          if (A(r, c) != 0) done = false;
        }
      A.check();
      if (done) {
        for (int i = 0; i < d; ++i) std::swap(A(i, piv), A(i, r));
        if (A(r, r) < 0)
          for (int i = 0; i < d; ++i) A(i, r) = -A(i, r);
        break;
      }
    }
  }
  for (int r = d - 1; r >= 0; --r)
    for (int c = r + 1; c < d; ++c) colop(c, r, fdiv128(A(r, c), A(r, r)));
  A.check();
  return A.narrowed();
}

void smith_normal_form(const IMat& M, IMat& Q, std::vector<i64>& eps, IMat& R, IMat& Uo, IMat& Vo) {
  const int d = M.d;
  BigMat A(M), U(IMat::identity(d)), V(IMat::identity(d));
  auto rowop = [&](int i, int j, i128 q) {  // row i -= q row j
    if (q == 0) return;
    for (int k = 0; k < d; ++k) {
      A(i, k) -= q * A(j, k);
      U(i, k) -= q * U(j, k);
    }
  };
  auto colop = [&](int i, int j, i128 q) {  // col i -= q col j
    if (q == 0) return;
    for (int k = 0; k < d; ++k) {
      A(k, i) -= q * A(k, j);
      V(k, i) -= q * V(k, j);
    }
  };
  auto rowswap = [&](int i, int j) {
    for (int k = 0; k < d; ++k) {
      std::swap(A(i, k), A(j, k));
      std::swap(U(i, k), U(j, k));
    }
  };
  auto colswap = [&](int i, int j) {
    for (int k = 0; k < d; ++k) {
      std::swap(A(k, i), A(k, j));
      std::swap(V(k, i), V(k, j));
    }
  };
  for (int t = 0; t < d; ++t) {
    for (int guard = 0;; ++guard) {
      if (guard > 100000) throw LatticeError{PFFT_ERR_OVERFLOW, "Smith form did not converge"};
      int bi = -1, bj = -1;
      for (int i = t; i < d; ++i)
        for (int j = t; j < d; ++j)
          if (A(i, j) != 0 && (bi < 0 || abs128(A(i, j)) < abs128(A(bi, bj)))) bi = i, bj = j;
      if (bi < 0) throw LatticeError{PFFT_ERR_SINGULAR, "singular matrix"};
      rowswap(t, bi);
      colswap(t, bj);
      bool clean = true;
      for (int i = t + 1; i < d; ++i) {
        rowop(i, t, fdiv128(A(i, t), A(t, t)));
        clean &= A(i, t) == 0;
      }
      for (int j = t + 1; j < d; ++j) {
        colop(j, t, fdiv128(A(t, j), A(t, t)));
        clean &= A(t, j) == 0;
      }
      A.check(); U.check(); V.check();
      if (!clean) continue;
      int badi = -1;
      for (int i = t + 1; i < d && badi < 0; ++i)
        for (int j = t + 1; j < d; ++j)
          if (A(i, j) % A(t, t) != 0) { badi = i; break; }
      if (badi >= 0) {
        rowop(t, badi, -1);  // row t += row badi, then re-reduce
        continue;
      }
      break;
    }
    if (A(t, t) < 0)
      for (int k = 0; k < d; ++k) {
        A(t, k) = -A(t, k);
        U(t, k) = -U(t, k);
      }
  }
  eps.assign(d, 0);
  for (int i = 0; i < d; ++i) eps[i] = narrow(A(i, i));
  Uo = U.narrowed();
  Vo = V.narrowed();
  if (!inverse_unimodular(Uo, Q) || !inverse_unimodular(Vo, R))
    throw LatticeError{PFFT_ERR_OVERFLOW, "Smith form transforms are not unimodular"};
}

void box_reduce(const IMat& H, i64* y) {
  for (int r = H.d - 1; r >= 0; --r) {
    i64 q = floordiv(y[r], H(r, r));
    if (q)
      for (int i = 0; i <= r; ++i) y[i] = narrow((i128)y[i] - (i128)q * H(i, r));
  }
}

i64 box_slot(const IMat& H, const i64* y) {
  i64 s = 0;
  for (int r = 0; r < H.d; ++r) s = s * H(r, r) + y[r];
  return s;
}

void box_point(const IMat& H, i64 slot, i64* y) {
  for (int r = H.d - 1; r >= 0; --r) {
    y[r] = slot % H(r, r);
    slot /= H(r, r);
  }
}

}  // namespace pfft
