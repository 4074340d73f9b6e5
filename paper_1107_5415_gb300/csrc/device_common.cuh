// Device helpers shared by the transform and split kernels: complex
// arithmetic, division by run-time invariant integers, small DFT butterflies
// and reduction of integer vectors into a Hermite box.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pfft {

// ---------------------------------------------------------------- complex
template <typename R>
struct CT;
template <>
struct CT<float> {
  using type = float2;
};
template <>
struct CT<double> {
  using type = double2;
};

// Load of data that another CTA of the same launch may have written (COH:
// through L2, bypassing the non-coherent L1 / read-only paths), or a plain
// load.
template <bool COH, typename T>
__device__ __forceinline__ T load_c(const T* p) {
  if constexpr (COH)
    return __ldcg(p);
  else
    return *p;
}

template <typename C>
__device__ __forceinline__ C cmake(decltype(C::x) a, decltype(C::x) b) {
  C c;
  c.x = a;
  c.y = b;
  return c;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C>
__device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
// multiply by -i
template <typename C>
__device__ __forceinline__ C cmul_mi(C a) { return cmake<C>(a.y, -a.x); }
template <typename C>
__device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmake<C>(a.x * s, a.y * s); }

// --------------------------------------------------- run-time invariant division
// Division of 0 <= n < 2^31 by a fixed divisor 1 <= d < 2^31 with one
// multiply-high, after Granlund & Montgomery, "Division by invariant integers
// using multiplication" (PLDI 1994): with l = ceil(log2 d) and
// mul = floor(2^32 (2^l - d) / d) + 1, n / d = (mulhi(n, mul) + n) >> l.
struct FastDiv {
  uint32_t d, mul, shift;
  __host__ void init(uint32_t dv) {
    d = dv;
    uint32_t l = 0;
    while ((uint64_t(1) << l) < dv) ++l;
    shift = l;
    mul = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - dv)) / dv + 1);
  }
  __device__ __forceinline__ int div(int n) const {
    uint32_t t = __umulhi(uint32_t(n), mul);
    return int((t + uint32_t(n)) >> shift);
  }
  __device__ __forceinline__ int mod(int n) const { return n - div(n) * int(d); }
};

// ------------------------------------------------------------ Hermite box
// Upper-triangular H (d <= 4) with row-major slot strides.  A point y of the
// box x_r [0, H_rr) is stored as int32 coordinates.
struct BoxDesc {
  int d;
  int H[4][4];
  int stride[4];
};

// Reduce y (each coordinate in [-2 H_rr, 3 H_rr)) into the box by
// subtracting / adding columns of H, last coordinate first.
__device__ __forceinline__ void box_fix(const BoxDesc& B, int* y) {
#pragma unroll
  for (int r = 3; r >= 0; --r) {
    if (r < B.d) {
      const int h = B.H[r][r];
      while (y[r] >= h) {
        y[r] -= h;
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (i < r) y[i] -= B.H[i][r];
      }
      while (y[r] < 0) {
        y[r] += h;
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (i < r) y[i] += B.H[i][r];
      }
    }
  }
}

// Slot of reduce(a + b) for two box points a, b (tables of d int32 each).
__device__ __forceinline__ int box_sum_slot(const BoxDesc& B, const int* a, const int* b) {
  int y[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) y[r] = (r < B.d) ? a[r] + b[r] : 0;
  box_fix(B, y);
  int s = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (r < B.d) s += y[r] * B.stride[r];
  return s;
}


// Slot of reduce(a + b) for two points a, b of the box, specialised on the
// dimension.  Coordinate r of the sum lies in [0, 2 H_rr); the corrections of
// the higher coordinates shift the lower ones by at most one diagonal each,
// so every coordinate needs a bounded number of conditional steps.
template <int DIM>
__device__ __forceinline__ int box_sum_slot_t(const BoxDesc& B, const int* a, const int* b) {
  if constexpr (DIM == 1) {
    int y = a[0] + b[0];
    if (y >= B.H[0][0]) y -= B.H[0][0];
    return y;
  } else if constexpr (DIM == 2) {
    int y1 = a[1] + b[1];
    const int c1 = y1 >= B.H[1][1];
    y1 -= c1 * B.H[1][1];
    int y0 = a[0] + b[0] - c1 * B.H[0][1];
    y0 += (y0 < 0) * B.H[0][0];
    y0 -= (y0 >= B.H[0][0]) * B.H[0][0];
    return y0 * B.stride[0] + y1;
  } else if constexpr (DIM == 3) {
    int y2 = a[2] + b[2];
    const int c2 = y2 >= B.H[2][2];
    y2 -= c2 * B.H[2][2];
    int y1 = a[1] + b[1] - c2 * B.H[1][2];
    int y0 = a[0] + b[0] - c2 * B.H[0][2];
    const int c1 = (y1 >= B.H[1][1]) - (y1 < 0);
    y1 -= c1 * B.H[1][1];
    y0 -= c1 * B.H[0][1];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      y0 += (y0 < 0) * B.H[0][0];
      y0 -= (y0 >= B.H[0][0]) * B.H[0][0];
    }
    return y0 * B.stride[0] + y1 * B.stride[1] + y2;
  } else {
    return box_sum_slot(B, a, b);
  }
}

// A table entry of a box point: TS = 2 (d <= 2) or 4 (d = 3, 4) int32,
// fetched with one vector load.
template <int TS>
__device__ __forceinline__ void load_point(const int* __restrict__ tab, int idx, int* y) {
  if constexpr (TS == 2) {
    const int2 v = __ldg(reinterpret_cast<const int2*>(tab) + idx);
    y[0] = v.x;
    y[1] = v.y;
    y[2] = 0;
    y[3] = 0;
  } else {
    const int4 v = __ldg(reinterpret_cast<const int4*>(tab) + idx);
    y[0] = v.x;
    y[1] = v.y;
    y[2] = v.z;
    y[3] = v.w;
  }
}

// ------------------------------------------------------------- butterflies
// In-register forward DFTs, X[k] = sum_n x[n] exp(-2 pi i n k / R).
template <typename C>
__device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <typename C>
__device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  C a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = cmul_mi(csub(x1, x3));
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, d);
  x3 = csub(b, d);
}

// exp(-2 pi i q / 16) for q = 0..15 (exact constants of cos/sin(pi/8 multiples)).
template <typename C>
__device__ __forceinline__ C w16(int q) {
  using R = decltype(C::x);
  const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173),
          h = R(0.70710678118654752440);
  switch (q & 15) {
    case 0: return cmake<C>(1, 0);
    case 1: return cmake<C>(c1, -s1);
    case 2: return cmake<C>(h, -h);
    case 3: return cmake<C>(s1, -c1);
    case 4: return cmake<C>(0, -1);
    case 5: return cmake<C>(-s1, -c1);
    case 6: return cmake<C>(-h, -h);
    case 7: return cmake<C>(-c1, -s1);
    case 8: return cmake<C>(-1, 0);
    case 9: return cmake<C>(-c1, s1);
    case 10: return cmake<C>(-h, h);
    case 11: return cmake<C>(-s1, c1);
    case 12: return cmake<C>(0, 1);
    case 13: return cmake<C>(s1, c1);
    case 14: return cmake<C>(h, h);
    default: return cmake<C>(c1, s1);
  }
}

// Length 8 as 4 x 2: n = 2 n1 + n2, k = k1 + 4 k2.
template <typename C>
__device__ __forceinline__ void dft8(C* x) {
  C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  o1 = cmul(o1, w16<C>(2));
  o2 = cmul_mi(o2);
  o3 = cmul(o3, w16<C>(6));
  x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
  x[1] = cadd(e1, o1); x[5] = csub(e1, o1);
  x[2] = cadd(e2, o2); x[6] = csub(e2, o2);
  x[3] = cadd(e3, o3); x[7] = csub(e3, o3);
}

// Length 16 as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.
template <typename C>
__device__ __forceinline__ void dft16(C* x) {
  C y[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C a = x[n2], b = x[4 + n2], c = x[8 + n2], d = x[12 + n2];
    dft4(a, b, c, d);  // over n1 -> k1
    y[n2 * 4 + 0] = a;
    y[n2 * 4 + 1] = (n2 == 0) ? b : cmul(b, w16<C>(n2));
    y[n2 * 4 + 2] = (n2 == 0) ? c : cmul(c, w16<C>(2 * n2));
    y[n2 * 4 + 3] = (n2 == 0) ? d : cmul(d, w16<C>(3 * n2));
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C a = y[k1], b = y[4 + k1], c = y[8 + k1], d = y[12 + k1];
    dft4(a, b, c, d);  // over n2 -> k2
    x[k1] = a;
    x[k1 + 4] = b;
    x[k1 + 8] = c;
    x[k1 + 12] = d;
  }
}

// Any length: direct sum with roots taken from a table of omega_N^t,
// omega_R^q = tab[q * (N / R)].
template <typename C, int R>
__device__ __forceinline__ void dft_direct(C* x, const C* __restrict__ tab, int step) {
  C w[R];
#pragma unroll
  for (int q = 0; q < R; ++q) w[q] = tab[q * step];
  C y[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    C acc = x[0];
#pragma unroll
    for (int n = 1; n < R; ++n) acc = cadd(acc, cmul(x[n], w[(n * k) % R]));
    y[k] = acc;
  }
#pragma unroll
  for (int k = 0; k < R; ++k) x[k] = y[k];
}

template <typename C, int R>
__device__ __forceinline__ void dft(C* x, const C* __restrict__ tab, int nD) {
  if constexpr (R == 2) {
    dft2(x[0], x[1]);
  } else if constexpr (R == 4) {
    dft4(x[0], x[1], x[2], x[3]);
  } else if constexpr (R == 8) {
    dft8(x);
  } else if constexpr (R == 16) {
    dft16(x);
  } else {
    dft_direct<C, R>(x, tab, nD / R);
  }
}

}  // namespace pfft
