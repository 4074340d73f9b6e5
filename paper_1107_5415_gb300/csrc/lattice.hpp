// Exact integer lattice algebra for the host planner (setup only).
//
// Notation follows Section 2.2: M a regular integer d x d matrix, m = |det M|,
// G(M) = Z^d / M Z^d, G(M^T) the frequency group, Smith normal form
// M = Q E R (eq. (SNF)), Hermite (pattern) normal form H = M U upper triangular
// (Section 6.1).  All arithmetic is exact (int64 storage, __int128 products);
// overflow is detected and reported instead of wrapping.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace pfft {

using i64 = int64_t;
using i128 = __int128;

struct IMat {
  int d = 0;
  std::vector<i64> a;  // row-major d*d
  IMat() = default;
  explicit IMat(int d_) : d(d_), a(size_t(d_) * d_, 0) {}
  i64& operator()(int i, int j) { return a[size_t(i) * d + j]; }
  i64 operator()(int i, int j) const { return a[size_t(i) * d + j]; }
  static IMat identity(int d);
  IMat transpose() const;
};

struct LatticeError {
  int code;  // pfft_status value
  std::string what;
};

IMat matmul(const IMat& A, const IMat& B);  // throws LatticeError on overflow
i64 determinant(const IMat& M);             // Bareiss, exact
IMat adjugate(const IMat& M);               // adj(M) M = det(M) I
bool inverse_unimodular(const IMat& U, IMat& inv);

// Column-style Hermite normal form: H = M U, H upper triangular,
// H_rr > 0, 0 <= H_rc < H_rr for c > r.  Unique.
IMat hermite_normal_form(const IMat& M);

// Smith normal form M = Q E R with Q, R unimodular and E = diag(eps),
// eps_j | eps_{j+1}.  Also returns U = Q^{-1}, V = R^{-1} (U M V = E).
void smith_normal_form(const IMat& M, IMat& Q, std::vector<i64>& eps, IMat& R, IMat& U, IMat& V);

// Representative of y mod H Z^d inside the box x_r [0, H_rr) (H upper triangular).
void box_reduce(const IMat& H, i64* y);
i64 box_slot(const IMat& H, const i64* y);
void box_point(const IMat& H, i64 slot, i64* y);

i64 floordiv(i64 a, i64 b);  // b > 0
i64 posmod(i64 a, i64 b);    // b > 0, result in [0, b)
i64 modinv(i64 a, i64 m);    // a invertible mod m
i64 gcd64(i64 a, i64 b);

}  // namespace pfft
