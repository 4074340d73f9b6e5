/*
 * CPU oracle for the pattern Fourier transform and the wavelet split step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a separate shared
 * library (liboracle) that only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load.  It shares no source, header, table or
 * helper with the GPU library.  Everything is plain FP64 with exact integer
 * phase numerators; there is no blocking or fast algorithm here.
 *
 * Transform (eq. (Fouriermatrix), Section 2.2):
 *     c_hat[k] = m^{-1/2} sum_{y in G(M)} c[y] exp(-2 pi i k^T M^{-1} y),
 * k running over G(M^T).  With M^{-1} = adj(M) / det(M), the phase is
 *     k^T M^{-1} y = n(k, y) / m  (mod 1),   n = sign(det M) * k^T adj(M) y  mod m,
 * an exact integer numerator.  Writing n = sum_r a_r y_r (a_r = sign * (k^T adj M)_r),
 * each term's phase is the product over coordinates of exp(-2 pi i (a_r y_r mod m)/m);
 * the sum itself is evaluated term by term over the input box in slot order.
 * The inverse uses the conjugate phase and the same m^{-1/2}.
 *
 * Wavelet split (Section 5.3, step 4, for |det J| = 2; symbols of Section 6.2):
 *   for g in G(N^T) with fibre {h0, h1} = {g, g + N^T l1} in G(M^T):
 *     d1[g] = 2^{-1/2} (conj(A(h0)) c[h0] + conj(A(h1)) c[h1])
 *     d2[g] = 2^{-1/2} (conj(B(h0)) c[h0] + conj(B(h1)) c[h1])
 *   B(h) = A(h + N^T l1) exp(-2 pi i h^T N^{-1} z), z the non-zero element of
 *   P(J) = Lambda(J) cap [-1/2,1/2)^d; h^T N^{-1} z = h^T M^{-1} (J z).
 *   Reconstruction inverts the 2x2 map per fibre:
 *     c[h] = sqrt(2) (A(h) d1[g] + B(h) d2[g]) / S,  S = |A(h0)|^2 + |A(h1)|^2,
 *   and the adjoint (conjugate transpose) is c[h] = 2^{-1/2} (A(h) d1 + B(h) d2).
 *
 * Scaling symbols, both as periodisations over the lattice J^T Z^d,
 *     w_B(t) = sum_{n in J^T Z^d} prod_j B(t_j + n_j),   t = N^{-T} h:
 *   DIRICHLET (Section 6.2): A(h) = sqrt(|det J| w(t)) with B the indicator of
 *     [-1/2, 1/2] taking 1/2 on the boundary, evaluated exactly in integers.
 *     Section 6.2 defines the symbol through c_k(phi_N) = A(h) c_k(phi_M),
 *     which presumes phi_N in V_M, i.e. [-1/2,1/2]^d inside J^T[-1/2,1/2]^d
 *     (true for the paper's dilations).  Where that holds, the periodised form
 *     equals the paper's case formula (kept below as DIRICHLET_CASE and
 *     pinned against it):  with k the representative of h in M^T[-1/2,1/2)^d,
 *       A(h) = 2^{(1 + r_M(k) - r_N(k))/2} if N^{-T} k in [-1/2,1/2]^d, else 0,
 *       r_X(k) = number of coordinates of X^{-T} k equal to +-1/2.
 *     For dilations without the containment the case formula breaks perfect
 *     reconstruction; the periodised form keeps it for every J.
 *   DLVP (not defined in the paper; the reading used by this project):
 *     A(h) = sqrt|det J| * w(t),  B(s) = clamp(((1+eta)/2 - |s|)/eta, 0, 1).
 *     PARITY UNPINNED beyond perfect reconstruction, the partition of unity on
 *     fibres and the eta -> 0 limit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

static int64_t floordiv128(i128 a, i128 b) { /* b > 0 */
  i128 q = a / b;
  if ((a % b) != 0 && a < 0) q -= 1;
  return (int64_t)q;
}
static int64_t mod128(i128 a, int64_t m) {
  i128 r = a % m;
  if (r < 0) r += m;
  return (int64_t)r;
}

/* Unravel a row-major slot index over the box x_r [0, ext_r). */
static void unravel(int d, const int64_t* ext, int64_t s, int64_t* v) {
  for (int r = d - 1; r >= 0; --r) {
    v[r] = s % ext[r];
    s /= ext[r];
  }
}

/* exp(sgn * 2 pi i n / m) for 0 <= n < m, straight from libm. */
static void unit_root(int64_t n, int64_t m, int sgn, double* re, double* im) {
  double a = 2.0 * M_PI * ((double)n / (double)m);
  *re = cos(a);
  *im = sgn * sin(a);
}

/*
 * Direct-sum transform.
 *   d, m, sdet        : dimension, |det M|, sign(det M)
 *   adjM              : adj(M), d*d row-major
 *   in_ext, out_ext   : diagonals of hnf(M) (input box) and hnf(M^T) (output box)
 *   batch             : number of signals; in is [batch][m] complex (re, im pairs)
 *   kslots, nk        : output slots to evaluate (NULL => all m, nk ignored)
 *   out               : [batch][nk] complex
 *   inverse           : 0 forward (exp(-...)), 1 inverse (exp(+...))
 *   Returns 0, or -1 on a bad argument.
 */
int po_transform(int d, int64_t m, int sdet, const int64_t* adjM, const int64_t* in_ext,
                 const int64_t* out_ext, int64_t batch, const double* in, double* out,
                 const int64_t* kslots, int64_t nk, int inverse, int nthreads) {
  if (d < 1 || d > 8 || m < 1 || batch < 1) return -1;
  if (!kslots) nk = m;
  int64_t fsum = 0;
  for (int r = 0; r < d; ++r) fsum += in_ext[r];
  const int sgn = inverse ? +1 : -1;
  const double scale = 1.0 / sqrt((double)m);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
  {
    double* f = (double*)malloc(sizeof(double) * 2 * (size_t)fsum);
    int64_t k[8], y[8], a[8];
#pragma omp for schedule(dynamic, 1)
    for (int64_t t = 0; t < nk; ++t) {
      int64_t ks = kslots ? kslots[t] : t;
      unravel(d, out_ext, ks, k);
      for (int r = 0; r < d; ++r) {
        i128 acc = 0;
        for (int i = 0; i < d; ++i) acc += (i128)k[i] * adjM[i * d + r];
        a[r] = mod128((i128)sdet * acc, m);
      }
      /* per-coordinate phase factors exp(sgn 2 pi i (a_r y_r mod m)/m) */
      double* fr = f;
      for (int r = 0; r < d; ++r) {
        for (int64_t v = 0; v < in_ext[r]; ++v) {
          int64_t n = (int64_t)(((i128)a[r] * v) % m);
          unit_root(n, m, sgn, &fr[2 * v], &fr[2 * v + 1]);
        }
        fr += 2 * in_ext[r];
      }
      for (int64_t b = 0; b < batch; ++b) {
        const double* x = in + 2 * b * m;
        double sre = 0.0, sim = 0.0;
        for (int r = 0; r < d; ++r) y[r] = 0;
        for (int64_t s = 0; s < m; ++s) {
          /* phase of term y: product of the coordinate factors */
          double pre = 1.0, pim = 0.0;
          const double* fq = f;
          for (int r = 0; r < d; ++r) {
            double qre = fq[2 * y[r]], qim = fq[2 * y[r] + 1];
            double tre = pre * qre - pim * qim;
            pim = pre * qim + pim * qre;
            pre = tre;
            fq += 2 * in_ext[r];
          }
          double xre = x[2 * s], xim = x[2 * s + 1];
          sre += xre * pre - xim * pim;
          sim += xre * pim + xim * pre;
          for (int r = d - 1; r >= 0; --r) { /* odometer, last coordinate fastest */
            if (++y[r] < in_ext[r]) break;
            y[r] = 0;
          }
        }
        out[2 * (b * nk + t)] = sre * scale;
        out[2 * (b * nk + t) + 1] = sim * scale;
      }
    }
    free(f);
  }
  return 0;
}

/* Representative of y mod H Z^d in the box of the upper-triangular H. */
static void box_reduce(int d, const int64_t* H, int64_t* y) {
  for (int r = d - 1; r >= 0; --r) {
    int64_t q = floordiv128(y[r], H[r * d + r]);
    if (q)
      for (int i = 0; i <= r; ++i) y[i] -= q * H[i * d + r];
  }
}

static int64_t slot_of(int d, const int64_t* H, const int64_t* y) {
  int64_t s = 0;
  for (int r = 0; r < d; ++r) s = s * H[r * d + r] + y[r];
  return s;
}

enum { PO_DIRICHLET = 0, PO_DLVP = 1, PO_DIRICHLET_CASE = 2 };

typedef struct {
  int d;
  const int64_t* adjMT; /* adj(M^T) */
  int64_t detM;
  const int64_t* J;
  const int64_t* adjJT; /* adj(J^T) */
  int64_t detJ;
  int symbol;
  double eta;
} symctx;

/* Scaling symbol A(h) for the class of h in G(M^T). */
static double scaling_symbol(const symctx* c, const int64_t* h) {
  const int d = c->d;
  const int64_t q = llabs(c->detM);
  const int sM = c->detM > 0 ? 1 : -1;
  int64_t u[8], v[8];
  /* M^{-T} h = adj(M^T) h / det M; centred numerators u in [-q/2, q/2) */
  for (int j = 0; j < d; ++j) {
    i128 p = 0;
    for (int i = 0; i < d; ++i) p += (i128)c->adjMT[j * d + i] * h[i];
    p *= sM;
    int64_t fl = floordiv128(2 * p + q, 2 * (i128)q);
    u[j] = (int64_t)(p - (i128)fl * q);
  }
  /* N^{-T} k = J^T M^{-T} k, numerators over q */
  for (int j = 0; j < d; ++j) {
    i128 s = 0;
    for (int i = 0; i < d; ++i) s += (i128)c->J[i * d + j] * u[i];
    v[j] = (int64_t)s;
  }
  if (c->symbol == PO_DIRICHLET_CASE) {
    int rM = 0, rN = 0;
    for (int j = 0; j < d; ++j) {
      if (2 * llabs(v[j]) > q) return 0.0;
      if (2 * llabs(u[j]) == q) ++rM;
      if (2 * llabs(v[j]) == q) ++rN;
    }
    return pow(2.0, 0.5 * (1 + rM - rN));
  }
  /* periodised weight: for each coordinate the shifts n with B(t_j + n) > 0,
   * t_j = v_j / q; Dirichlet weights decided on exact integer numerators */
  const double eta = c->eta;
  double wts[8][6];
  int64_t nval[8][6];
  int nc[8];
  for (int j = 0; j < d; ++j) {
    nc[j] = 0;
    const int64_t n0 = floordiv128(-(i128)v[j], q);
    for (int64_t n = n0 - 2; n <= n0 + 3; ++n) {
      const i128 a = (i128)v[j] + (i128)n * q; /* numerator of t_j + n */
      const i128 aa = a < 0 ? -a : a;
      double b;
      if (c->symbol == PO_DIRICHLET) {
        b = (2 * aa < q) ? 1.0 : (2 * aa == q) ? 0.5 : 0.0;
      } else {
        b = ((1.0 + eta) / 2.0 - (double)aa / (double)q) / eta;
        if (b > 1.0) b = 1.0;
      }
      if (b <= 0.0) continue;
      wts[j][nc[j]] = b;
      nval[j][nc[j]] = n;
      ++nc[j];
    }
    if (nc[j] == 0) return 0.0;
  }
  int idx[8] = {0};
  double w = 0.0;
  const int64_t aJ = llabs(c->detJ);
  for (;;) {
    int member = 1; /* n in J^T Z^d  <=>  adj(J^T) n = 0 mod |det J| */
    for (int i = 0; i < d && member; ++i) {
      i128 s = 0;
      for (int j = 0; j < d; ++j) s += (i128)c->adjJT[i * d + j] * nval[j][idx[j]];
      if (mod128(s, aJ) != 0) member = 0;
    }
    if (member) {
      double p = 1.0;
      for (int j = 0; j < d; ++j) p *= wts[j][idx[j]];
      w += p;
    }
    int j = d - 1;
    while (j >= 0 && ++idx[j] == nc[j]) idx[j--] = 0;
    if (j < 0) break;
  }
  if (c->symbol == PO_DIRICHLET) return sqrt((double)aJ * w);
  return sqrt((double)aJ) * w;
}

/* exp(-2 pi i h^T M^{-1} u) with the exact numerator sign(det M) h^T adj(M) u mod |det M|. */
static void wavelet_phase(const symctx* c, const int64_t* h, const int64_t* u, double* re,
                          double* im) {
  const int d = c->d;
  const int64_t q = llabs(c->detM);
  i128 s = 0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) s += (i128)h[i] * c->adjMT[j * d + i] * u[j]; /* adj(M)=adj(M^T)^T */
  if (c->detM < 0) s = -s;
  unit_root(mod128(s, q), q, -1, re, im);
}

/*
 * One level of the wavelet split (mode 0), its inverse (mode 1: reconstruct)
 * or its adjoint (mode 2).  Arrays are complex (re, im pairs):
 *   chat : [batch][mM]  coefficients on G(M^T), box of hnf(M^T) = HM
 *   d1,d2: [batch][mN]  scaling / wavelet parts on G(N^T), box of hnf(N^T) = HN
 *   NTl1 : N^T l1 for the non-zero class l1 of G(J^T);  u = J z.
 */
int po_wavelet_level(int d, const int64_t* HM, const int64_t* HN, const int64_t* adjMT,
                     int64_t detM, const int64_t* J, const int64_t* adjJT, int64_t detJ,
                     const int64_t* NTl1, const int64_t* u, int symbol, double eta,
                     int64_t batch, int mode, double* chat, double* d1, double* d2,
                     int nthreads) {
  if (d < 1 || d > 8 || llabs(detJ) != 2) return -1;
  if (symbol < PO_DIRICHLET || symbol > PO_DIRICHLET_CASE) return -1;
  if (symbol == PO_DLVP && !(eta > 0.0 && eta < 1.0)) return -1;
  int64_t mM = 1, mN = 1, ext[8];
  for (int r = 0; r < d; ++r) {
    mM *= HM[r * d + r];
    mN *= HN[r * d + r];
    ext[r] = HN[r * d + r];
  }
  if (mM != 2 * mN) return -1;
  symctx c = {d, adjMT, detM, J, adjJT, detJ, symbol, eta};
  const double r2 = sqrt(2.0);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(static)
  for (int64_t gs = 0; gs < mN; ++gs) {
    int64_t g[8], h0[8], h1[8];
    unravel(d, ext, gs, g);
    for (int r = 0; r < d; ++r) {
      h0[r] = g[r];
      h1[r] = g[r] + NTl1[r];
    }
    box_reduce(d, HM, h0);
    box_reduce(d, HM, h1);
    const int64_t s0 = slot_of(d, HM, h0), s1 = slot_of(d, HM, h1);
    const double A0 = scaling_symbol(&c, h0), A1 = scaling_symbol(&c, h1);
    double e0r, e0i, e1r, e1i;
    wavelet_phase(&c, h0, u, &e0r, &e0i);
    wavelet_phase(&c, h1, u, &e1r, &e1i);
    /* B(h0) = A(h1) e(h0), B(h1) = A(h0) e(h1) */
    const double B0r = A1 * e0r, B0i = A1 * e0i, B1r = A0 * e1r, B1i = A0 * e1i;
    const double S = A0 * A0 + A1 * A1;
    for (int64_t b = 0; b < batch; ++b) {
      double* C = chat + 2 * b * mM;
      double* D1 = d1 + 2 * b * mN;
      double* D2 = d2 + 2 * b * mN;
      if (mode == 0) {
        const double c0r = C[2 * s0], c0i = C[2 * s0 + 1], c1r = C[2 * s1], c1i = C[2 * s1 + 1];
        D1[2 * gs] = (A0 * c0r + A1 * c1r) / r2;
        D1[2 * gs + 1] = (A0 * c0i + A1 * c1i) / r2;
        /* conj(B) c */
        D2[2 * gs] = (B0r * c0r + B0i * c0i + B1r * c1r + B1i * c1i) / r2;
        D2[2 * gs + 1] = (B0r * c0i - B0i * c0r + B1r * c1i - B1i * c1r) / r2;
      } else {
        const double fac = (mode == 1) ? r2 / S : 1.0 / r2;
        const double ar = D1[2 * gs], ai = D1[2 * gs + 1], br = D2[2 * gs], bi = D2[2 * gs + 1];
        C[2 * s0] = fac * (A0 * ar + B0r * br - B0i * bi);
        C[2 * s0 + 1] = fac * (A0 * ai + B0r * bi + B0i * br);
        C[2 * s1] = fac * (A1 * ar + B1r * br - B1i * bi);
        C[2 * s1 + 1] = fac * (A1 * ai + B1r * bi + B1i * br);
      }
    }
  }
  return 0;
}

/* Scaling symbol values for a list of classes (for the oracle's own tests). */
int po_scaling_symbol(int d, const int64_t* adjMT, int64_t detM, const int64_t* J,
                      const int64_t* adjJT, int64_t detJ, int symbol, double eta,
                      int64_t n, const int64_t* hs, double* out) {
  symctx c = {d, adjMT, detM, J, adjJT, detJ, symbol, eta};
  for (int64_t t = 0; t < n; ++t) out[t] = scaling_symbol(&c, hs + t * d);
  return 0;
}
