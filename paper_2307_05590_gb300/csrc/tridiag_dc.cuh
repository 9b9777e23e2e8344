// Eigen-decomposition of a real symmetric tridiagonal matrix by divide and conquer (Cuppen's
// method with the stable eigenvector formula of Gu and Eisenstat), one CTA per matrix, for the
// Hermitian-pencil preparation: T = Z Lambda Z^T with Z orthonormal, for n <= MROM_MAX_R.
//
// The matrix is torn at every multiple of kDcLeaf (T = blockdiag(T_1', T_2', ...) + sum rho v v^T
// with the diagonal entries next to each split lowered by |rho|), the leaves (<= kDcLeaf rows) are
// diagonalised by cyclic Jacobi in registers, one thread per leaf, and neighbouring blocks are
// merged level by level, every merge of a level in parallel.  A merge of blocks with eigenpairs
// (D_1, Q_1), (D_2, Q_2) coupled by rho v v^T is the rank-one problem D + rho z z^T with
// z = [last row of Q_1, sign(rho) first row of Q_2]:
//   - the eigenvalues are sorted with z (ranks by counting);
//   - deflation: entries with rho |z_i| <= tol keep (d_i, e_i); two remaining entries with
//     |d_i - d_j| <= tol are rotated so that z_j = 0 (the rotation is applied to Q's columns);
//   - the k remaining roots of the secular equation 1 + rho sum z_i^2 / (d_i - lambda) = 0, one in
//     each interval (d_i, d_i+1) and one in (d_k, d_k + rho |z|^2), are found on
//     lambda = d_o + tau, the origin d_o being the nearer pole, so that every difference
//     d_i - lambda = (d_i - d_o) - tau is accurate: a single-precision bisection gives the start,
//     a two-pole rational interpolation safeguarded by bisection finishes in double precision
//     (about 2.4 double-precision evaluations per root on pencil tridiagonals);
//   - z is recomputed from the roots (Loewner's formula, z^_i^2 = prod_j (lambda_j - d_i) /
//     (rho prod_{j!=i} (d_j - d_i)), as products of ratios of order one), which makes the
//     eigenvectors u_j = (z^_i / (d_i - lambda_j))_i / norm orthogonal to working precision;
//   - Q <- Q P U for the block (one float64 GEMM, n x k x k); Q is block diagonal in the two
//     halves except for columns that a deflation rotation mixed, so a row of the upper half sums
//     only over the kept columns with entries there (and likewise the lower half): the terms
//     skipped are exact zeros, and about half of the GEMM's multiplications go.
// tol = 8 eps max(max|d|, rho max z^2).  Q lives in global memory (L2-resident workspace), per-
// position data in shared memory.  A non-finite value clears *ok (the caller then routes the
// object elsewhere); every loop is bounded.
#pragma once

#include <cfloat>
#include <cmath>

namespace mrom {
namespace dc {

constexpr int kDcLeaf = 4;          // leaf size (cyclic Jacobi in registers)
constexpr int kDcMaxIter = 128;     // double-precision steps per secular root (bound)
constexpr int kDcMaxN = MROM_MAX_R;

// Shared-memory state of one decomposition (per-position arrays of length n <= kDcMaxN).
struct DcShared {
  double d0[kDcMaxN];      // torn diagonal
  double lam[kDcMaxN];     // eigenvalue of each column of Q (current level)
  double ds[kDcMaxN];      // sorted eigenvalues of each merge (then deflation-modified)
  double zs[kDcMaxN];      // z in sorted order (then deflation-modified)
  double tau[kDcMaxN];     // root offsets (per kept index)
  double zh[kDcMaxN];      // Loewner z (per kept index)
  double cn[kDcMaxN];      // 1 / column norms of U (per kept index)
  double rc[kDcMaxN];      // deflation rotations (c, s) per merge, at the merge's offset
  double rs[kDcMaxN];
  int perm[kDcMaxN];       // sorted position -> column offset within the merge
  int ty[kDcMaxN];         // rows with entries in the column at a sorted position: 1 upper, 2 lower
  int klist[2 * kDcMaxN];  // per merge at 2 a: kept indices with upper rows, then (at 2 a + nmg) lower
  int kcol[2 * kDcMaxN];   // their column offsets within the merge
  int keep[kDcMaxN];       // kept sorted positions, per merge at its offset
  int kinv[kDcMaxN];       // sorted position -> kept index (or -1)
  int org[kDcMaxN];        // root origin (kept index of the pole), per kept index
  int rpair[2 * kDcMaxN];  // deflation rotation column pairs (sorted positions)
  int nk[kDcMaxN / 2 + 1]; // kept count per merge
  int nrot[kDcMaxN / 2 + 1];
  int nk1[kDcMaxN / 2 + 1];  // kept columns with entries in the upper rows, per merge
  int nk2[kDcMaxN / 2 + 1];  // ... in the lower rows
  double rho[kDcMaxN / 2 + 1];
  int bad;
};

// Cyclic Jacobi on a symmetric tridiagonal leaf of size m <= kDcLeaf (d, e in registers):
// eigenvalues w and eigenvectors V (columns).
__device__ inline void leaf_jacobi(int m, const double* d, const double* e, double (&w)[kDcLeaf],
                                   double (&V)[kDcLeaf][kDcLeaf]) {
  double a[kDcLeaf][kDcLeaf];
#pragma unroll
  for (int i = 0; i < kDcLeaf; ++i)
#pragma unroll
    for (int j = 0; j < kDcLeaf; ++j) {
      a[i][j] = 0.0;
      V[i][j] = i == j ? 1.0 : 0.0;
    }
#pragma unroll
  for (int i = 0; i < kDcLeaf; ++i) {
    if (i < m) a[i][i] = d[i];
    if (i + 1 < kDcLeaf && i + 1 < m) a[i][i + 1] = a[i + 1][i] = e[i];
  }
  double fro = 0.0;
#pragma unroll
  for (int i = 0; i < kDcLeaf; ++i)
#pragma unroll
    for (int j = 0; j < kDcLeaf; ++j) fro = fma(a[i][j], a[i][j], fro);
  for (int sweep = 0; sweep < 16; ++sweep) {
    double off = 0.0;
#pragma unroll
    for (int i = 0; i < kDcLeaf; ++i)
#pragma unroll
      for (int j = i + 1; j < kDcLeaf; ++j) off = fma(a[i][j], a[i][j], off);
    if (!(2.0 * off > DBL_EPSILON * DBL_EPSILON * fro)) break;
#pragma unroll
    for (int p = 0; p < kDcLeaf; ++p)
#pragma unroll
      for (int q = p + 1; q < kDcLeaf; ++q) {
        const double apq = a[p][q];
        if (apq == 0.0) continue;
        const double th = (a[q][q] - a[p][p]) / (2.0 * apq);
        const double t = fabs(th) > 1e150 ? 0.5 / th : (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(fma(th, th, 1.0)));
        const double c = 1.0 / sqrt(fma(t, t, 1.0)), s = t * c;
#pragma unroll
        for (int k = 0; k < kDcLeaf; ++k) {  // rows p, q then columns p, q of a
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < kDcLeaf; ++k) {
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
#pragma unroll
        for (int k = 0; k < kDcLeaf; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
#pragma unroll
  for (int i = 0; i < kDcLeaf; ++i) w[i] = a[i][i];
}

// Root of the secular equation 1 + rho sum_j z_j^2 / (d_j - lambda) = 0 with index i of the k kept
// entries (sorted d): lambda = d_o + tau.  The bracket is narrowed in single precision first
// (cheap divisions), then a rational interpolation with the bisection safeguard finishes in double
// precision; both bounded.
template <class DK, class ZK>
__device__ inline void secular_root(int i, int k, double rho, DK dk, ZK zk, int& o_out, double& tau_out) {
  double lo, hi;
  int o;
  if (i < k - 1) {
    const double di = dk(i), mid = 0.5 * (dk(i + 1) - di);
    double f = 1.0;
    for (int j = 0; j < k; ++j) {
      const double zj = zk(j);
      f += rho * zj * zj / ((dk(j) - di) - mid);
    }
    if (f >= 0.0) {
      o = i; lo = 0.0; hi = mid;
    } else {
      o = i + 1; lo = -mid; hi = 0.0;
    }
  } else {
    double zz = 0.0;
    for (int j = 0; j < k; ++j) zz = fma(zk(j), zk(j), zz);
    o = k - 1; lo = 0.0; hi = rho * zz;
  }
  const double dorg = dk(o);
  // f(tau) = 1 + rho sum z_j^2 / ((d_j - d_o) - tau) increases on (lo, hi); f(lo+) < 0 < f(hi-)
  // (the bracket ends are a pole and the midpoint, or the last pole and d_k + rho |z|^2)
  if (k == 1) {  // f = 1 - rho z^2 / tau: the root is the bracket's upper end
    o_out = o;
    tau_out = hi;
    return;
  }
  // the two poles that enclose the root (for the last root: the last two poles); f = 1 + psi + phi
  // with psi the terms of the poles up to P and phi the rest
  const int P = i < k - 1 ? i : k - 2;
  const double dP = dk(P) - dorg, dQ = dk(P + 1) - dorg;
  auto eval = [&](double t, double& psi, double& dpsi, double& phi, double& dphi) {
    psi = dpsi = phi = dphi = 0.0;
    for (int j = 0; j <= P; ++j) {
      const double q = zk(j) / ((dk(j) - dorg) - t);
      psi = fma(rho * zk(j), q, psi);
      dpsi = fma(rho * q, q, dpsi);
    }
    for (int j = P + 1; j < k; ++j) {
      const double q = zk(j) / ((dk(j) - dorg) - t);
      phi = fma(rho * zk(j), q, phi);
      dphi = fma(rho * q, q, dphi);
    }
  };
  // single-precision bisection to about 1e-6 of the bracket (24 halvings at most) gives the
  // starting point; the double-precision iteration keeps the full bracket as its safeguard (single
  // precision may misjudge the sign next to the root, so its bracket is not trusted)
  double tau;
  {
    float a = (float)lo, b = (float)hi;
    for (int it = 0; it < 24 && b - a > 1e-6f * fmaxf(fabsf(a), fabsf(b)); ++it) {
      const float t = 0.5f * (a + b);
      float f = 1.0f;
      for (int j = 0; j < k; ++j) {
        const float zj = (float)zk(j);
        f += (float)rho * zj * zj / ((float)(dk(j) - dorg) - t);
      }
      if (f < 0.0f) a = t; else b = t;
    }
    tau = 0.5 * ((double)a + (double)b);
    if (!(tau > lo && tau < hi)) tau = 0.5 * (lo + hi);
  }
  // Rational interpolation in double precision: psi and phi are each replaced by a constant plus
  // one pole term at their own enclosing pole, matching value and slope at tau (the "middle way" of
  // R.-C. Li, "Solving secular equations stably and efficiently", LAPACK Working Note 89, 1993);
  // the model's root in the bracket is the next iterate.  Converges quadratically, and from either
  // side of a root next to a pole, where Newton's tangent on f itself overshoots.  Steps outside
  // the (sign-updated) bracket fall back to bisection.
  for (int it = 0; it < kDcMaxIter; ++it) {
    double psi, dpsi, phi, dphi;
    eval(tau, psi, dpsi, phi, dphi);
    const double f = 1.0 + psi + phi;
    // stop at the rounding level of f (a few ulps of the absolute sum of its terms, which is
    // 1 + phi - psi as the terms of psi are negative and those of phi positive; one ulp of tau moves
    // f by |tau| f')
    if (fabs(f) <= DBL_EPSILON * (4.0 * (1.0 + phi - psi) + fabs(tau) * (dpsi + dphi))) break;
    if (f < 0.0) lo = tau; else hi = tau;
    const double D1 = dP - tau, D2 = dQ - tau;
    const double b1 = dpsi * D1 * D1, b2 = dphi * D2 * D2;
    const double C = 1.0 + (psi - dpsi * D1) + (phi - dphi * D2);
    // C (D1 - eta)(D2 - eta) + b1 (D2 - eta) + b2 (D1 - eta) = 0
    const double Aq = C * (D1 + D2) + b1 + b2, Bq = f * D1 * D2;
    const double sq = sqrt(fmax(0.0, Aq * Aq - 4.0 * C * Bq)), s = Aq + copysign(sq, Aq);
    double tn = 0.5 * (lo + hi);
    if (s != 0.0) {
      const double e1 = 2.0 * Bq / s;  // the root of smaller magnitude
      if (tau + e1 > lo && tau + e1 < hi) {
        tn = tau + e1;
      } else if (C != 0.0) {
        const double e2 = s / (2.0 * C);
        if (tau + e2 > lo && tau + e2 < hi) tn = tau + e2;
      }
    }
    const bool done = fabs(tn - tau) <= 2.0 * DBL_EPSILON * fabs(tn) || hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi));
    tau = tn;
    if (done) break;
  }
  if (tau == 0.0) tau = (o == i ? 1.0 : -1.0) * DBL_MIN;  // never exactly on the pole
  o_out = o;
  tau_out = tau;
}

// Z Lambda Z^T = T for the symmetric tridiagonal (dg, eg) (eg[i] couples i and i + 1), n <= kDcMaxN.
// A, B, U: n x n float64 global workspace (row-major).  Returns the buffer (A or B) that holds
// Z (column j is the eigenvector of S.lam[j]); S.bad != 0 after a non-finite value.  All NT
// threads of the CTA call it.
template <int NT>
__device__ double* tridiag_dc(const double* __restrict__ dg, const double* __restrict__ eg, int n,
                              double* __restrict__ A, double* __restrict__ B, double* __restrict__ U,
                              DcShared& S) {
  const int tid = threadIdx.x;
  if (tid == 0) S.bad = 0;
  // torn diagonal: the rows next to every split at a multiple of kDcLeaf lose |e| there
  for (int i = tid; i < n; i += NT) {
    double di = dg[i];
    if (i > 0 && i % kDcLeaf == 0) di -= fabs(eg[i - 1]);
    if (i + 1 < n && (i + 1) % kDcLeaf == 0) di -= fabs(eg[i]);
    S.d0[i] = di;
  }
  for (int idx = tid; idx < n * n; idx += NT) {
    A[idx] = 0.0;
    B[idx] = 0.0;
  }
  __syncthreads();
  // leaves
  for (int l = tid; l * kDcLeaf < n; l += NT) {
    const int a = l * kDcLeaf, m = min(kDcLeaf, n - a);
    double dd[kDcLeaf], ee[kDcLeaf], w[kDcLeaf], V[kDcLeaf][kDcLeaf];
#pragma unroll
    for (int i = 0; i < kDcLeaf; ++i) {
      dd[i] = i < m ? S.d0[a + i] : 0.0;
      ee[i] = i + 1 < m ? eg[a + i] : 0.0;
    }
    leaf_jacobi(m, dd, ee, w, V);
#pragma unroll
    for (int i = 0; i < kDcLeaf; ++i) {
      if (i < m) {
        S.lam[a + i] = w[i];
#pragma unroll
        for (int j = 0; j < kDcLeaf; ++j)
          if (j < m) A[(size_t)(a + i) * n + a + j] = V[i][j];
      }
    }
  }
  __syncthreads();
  double* Q = A;
  double* Qn = B;
  for (int bs = kDcLeaf; bs < n; bs *= 2) {
    const int span = 2 * bs;
    const int nm = (n + span - 1) / span;
    // (1) z of every merge in column order (S.zh as scratch); ranks of the eigenvalues
    for (int p = tid; p < n; p += NT) {
      const int a = (p / span) * span, nmg = min(span, n - a);
      if (nmg <= bs) continue;  // a lone block is carried over
      const int s = a + bs, c = p - a;
      const double ev = eg[s - 1];
      S.zh[p] = c < bs ? Q[(size_t)(s - 1) * n + p] : (ev < 0.0 ? -Q[(size_t)s * n + p] : Q[(size_t)s * n + p]);
    }
    __syncthreads();
    for (int p = tid; p < n; p += NT) {
      const int a = (p / span) * span, nmg = min(span, n - a);
      if (nmg <= bs) continue;
      const double lp = S.lam[p];
      int rank = 0;
      for (int q = a; q < a + nmg; ++q) {
        const double lq = S.lam[q];
        rank += (lq < lp || (lq == lp && q < p)) ? 1 : 0;
      }
      S.perm[a + rank] = p - a;
    }
    __syncthreads();
    for (int p = tid; p < n; p += NT) {
      const int a = (p / span) * span, nmg = min(span, n - a);
      if (nmg <= bs) continue;
      S.ds[p] = S.lam[a + S.perm[p]];
      S.zs[p] = S.zh[a + S.perm[p]];
    }
    __syncthreads();
    // (2) deflation, one thread per merge (sequential over its sorted entries)
    for (int mi = tid; mi < nm; mi += NT) {
      const int a = mi * span, nmg = min(span, n - a);
      if (nmg <= bs) continue;
      const double rho = fabs(eg[a + bs - 1]);
      double dmax = 0.0, zmax = 0.0;
      for (int p = a; p < a + nmg; ++p) {
        dmax = fmax(dmax, fabs(S.ds[p]));
        zmax = fmax(zmax, fabs(S.zs[p]));
      }
      const double tol = 8.0 * DBL_EPSILON * fmax(dmax, rho * zmax * zmax);
      for (int p = a; p < a + nmg; ++p) S.ty[p] = S.perm[p] < bs ? 1 : 2;
      int last = -1, nr = 0;
      for (int p = a; p < a + nmg; ++p) {
        S.kinv[p] = 0;
        if (rho * fabs(S.zs[p]) <= tol) {
          S.kinv[p] = -1;
          continue;
        }
        if (last >= 0 && S.ds[p] - S.ds[last] <= tol) {
          const double zl = S.zs[last], zp = S.zs[p];
          const double r = hypot(zl, zp), c = zl / r, sn = zp / r;
          const double dl = S.ds[last], dp = S.ds[p];
          S.ds[last] = fma(dl * c, c, dp * sn * sn);
          S.ds[p] = fma(dl * sn, sn, dp * c * c);
          S.zs[last] = r;
          S.zs[p] = 0.0;
          S.kinv[p] = -1;
          S.rc[a + nr] = c;
          S.rs[a + nr] = sn;
          S.rpair[2 * (a + nr)] = last;
          S.rpair[2 * (a + nr) + 1] = p;
          S.ty[last] |= S.ty[p];  // the rotation mixes the two columns' rows
          ++nr;
        } else {
          last = p;
        }
      }
      int k = 0;
      for (int p = a; p < a + nmg; ++p)
        if (S.kinv[p] >= 0) {
          S.keep[a + k] = p;
          S.kinv[p] = k++;
        }
      int n1 = 0, n2 = 0;
      for (int i = 0; i < k; ++i) {
        const int sp = S.keep[a + i], t = S.ty[sp];
        if (t & 1) {
          S.klist[2 * a + n1] = i;
          S.kcol[2 * a + n1++] = S.perm[sp];
        }
        if (t & 2) {
          S.klist[2 * a + nmg + n2] = i;
          S.kcol[2 * a + nmg + n2++] = S.perm[sp];
        }
      }
      S.nk[mi] = k;
      S.nk1[mi] = n1;
      S.nk2[mi] = n2;
      S.nrot[mi] = nr;
      S.rho[mi] = rho;
    }
    __syncthreads();
    // (3) the deflation rotations on Q's columns (in order; rows are independent)
    for (int p = tid; p < n; p += NT) {
      const int mi = p / span, a = mi * span, nmg = min(span, n - a);
      if (nmg <= bs) continue;
      double* row = Q + (size_t)p * n + a;
      for (int t = 0; t < S.nrot[mi]; ++t) {
        const int ca = S.perm[S.rpair[2 * (a + t)]], cb = S.perm[S.rpair[2 * (a + t) + 1]];
        const double c = S.rc[a + t], sn = S.rs[a + t];
        const double qa = row[ca], qb = row[cb];
        row[ca] = fma(c, qa, sn * qb);
        row[cb] = fma(c, qb, -sn * qa);
      }
    }
    // (4) secular roots, one thread per kept entry
    for (int p = tid; p < n; p += NT) {
      const int mi = p / span, a = mi * span, nmg = min(span, n - a);
      if (nmg <= bs) continue;
      const int i = p - a, k = S.nk[mi];
      if (i >= k) continue;
      const int* kp = S.keep + a;
      auto dk = [&](int j) { return S.ds[kp[j]]; };
      auto zk = [&](int j) { return S.zs[kp[j]]; };
      int o;
      double tau;
      secular_root(i, k, S.rho[mi], dk, zk, o, tau);
      S.org[p] = o;
      S.tau[p] = tau;
    }
    __syncthreads();
    // (5) Loewner's z: z^_i^2 = -(d_i - lam_i) / rho * prod_{j != i} (d_i - lam_j) / (d_i - d_j)
    for (int p = tid; p < n; p += NT) {
      const int mi = p / span, a = mi * span, nmg = min(span, n - a);
      if (nmg <= bs) continue;
      const int i = p - a, k = S.nk[mi];
      if (i >= k) continue;
      const int* kp = S.keep + a;
      const double di = S.ds[kp[i]];
      double w = -((di - S.ds[kp[S.org[a + i]]]) - S.tau[a + i]) / S.rho[mi];
      for (int j = 0; j < k; ++j) {
        if (j == i) continue;
        const double dij = (di - S.ds[kp[S.org[a + j]]]) - S.tau[a + j];
        w *= dij / (di - S.ds[kp[j]]);
      }
      S.zh[p] = copysign(sqrt(fabs(w)), S.zs[kp[i]]);
    }
    __syncthreads();
    // (6) U = (z^_i / (d_i - lam_j)) with unit columns (U at the merge's diagonal block)
    for (int p = tid; p < n; p += NT) {
      const int mi = p / span, a = mi * span, nmg = min(span, n - a);
      if (nmg <= bs) continue;
      const int j = p - a, k = S.nk[mi];
      if (j >= k) continue;
      const int* kp = S.keep + a;
      const double dorg = S.ds[kp[S.org[p]]], tj = S.tau[p];
      double nrm = 0.0;
      for (int i = 0; i < k; ++i) {
        const double u = S.zh[a + i] / ((S.ds[kp[i]] - dorg) - tj);
        U[(size_t)(a + i) * n + a + j] = u;
        nrm = fma(u, u, nrm);
      }
      S.cn[p] = 1.0 / sqrt(nrm);
      if (!isfinite(S.cn[p])) atomicOr(&S.bad, 1);
    }
    __syncthreads();
    // (7) Qn = Q P U on the merge's block; new eigenvalues
    for (int idx = tid; idx < n * span; idx += NT) {
      const int p = idx / span, c = idx - (idx / span) * span;  // row p, column offset c
      const int mi = p / span, a = mi * span, nmg = min(span, n - a);
      if (c >= nmg) continue;
      double v, lamv = 0.0;
      if (nmg <= bs) {  // lone block
        v = Q[(size_t)p * n + a + c];
        lamv = S.lam[a + c];
      } else {
        const int sp = a + c, j = S.kinv[sp];
        if (j < 0) {
          v = Q[(size_t)p * n + a + S.perm[sp]];
          lamv = S.ds[sp];
        } else {
          const int* kp = S.keep + a;
          const double* qrow = Q + (size_t)p * n + a;
          const bool up = p - a < bs;  // the half of the merge that row p lies in
          const int nl = up ? S.nk1[mi] : S.nk2[mi], l0 = 2 * a + (up ? 0 : nmg);
          double acc = 0.0;
          for (int t = 0; t < nl; ++t)
            acc = fma(qrow[S.kcol[l0 + t]], U[(size_t)(a + S.klist[l0 + t]) * n + a + j], acc);
          v = acc * S.cn[a + j];
          lamv = S.ds[kp[S.org[a + j]]] + S.tau[a + j];
        }
      }
      Qn[(size_t)p * n + a + c] = v;
      if (p == a) S.d0[a + c] = lamv;  // staged in d0 (free after the leaves)
    }
    __syncthreads();
    for (int p = tid; p < n; p += NT) S.lam[p] = S.d0[p];
    double* t = Q;
    Q = Qn;
    Qn = t;
    __syncthreads();
  }
  for (int p = tid; p < n; p += NT)
    if (!isfinite(S.lam[p])) atomicOr(&S.bad, 1);
  __syncthreads();
  return Q;
}

}  // namespace dc
}  // namespace mrom
