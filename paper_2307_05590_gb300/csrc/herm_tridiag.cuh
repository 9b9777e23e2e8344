// Hermitian tridiagonalisation (Householder) and implicit QL for the pencil preparation and the
// snapshot eigensolver: herm_tridiag on a full matrix in any memory (snapshot Grams up to
// MROM_MAX_SNAPSHOTS), herm_tridiag_packed on a packed lower triangle in shared memory (the
// pencil's H, r <= MROM_MAX_R), both finished by accumulate_q1.  Device code only; one CTA of NT
// threads.
#pragma once

#include <cfloat>
#include <cuda_runtime.h>

namespace mrom {
namespace hq {

__device__ __forceinline__ double2 cmac(double2 c, double2 a, double2 b) {  // c + a b
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cmacc(double2 c, double2 a, double2 b) {  // c + conj(a) b
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}

// CTA-wide sum of one value per thread (every thread gets the result; fixed order).
template <int NT>
__device__ double blk_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NT / 32; ++k) s += red[k];
  __syncthreads();
  return s;
}

// Row and column of entry e of a packed lower triangle (row i holds columns 0..i):
// e = i (i + 1) / 2 + j.  Float square root, then exact integer correction.
__device__ __forceinline__ void tri_rc(int e, int& i, int& j) {
  int t = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (t * (t + 1) / 2 > e) --t;
  while ((t + 1) * (t + 2) / 2 <= e) ++t;
  i = t;
  j = e - t * (t + 1) / 2;
}

// Q1 = P_0 P_1 ... P_{r-3} from the reflectors left by a Householder reduction (vat(k, i) = entry i of
// the vector of step k, tau in stau), accumulated backwards on the trailing block; then the phases
// D_0 = 1, D_{k+1} = D_k e_k / |e_k| that make D^H T D real with off-diagonal |e_k| (se), and
// Q = Q1 D.  Scratch (shared): sph (r entries), part (NT entries).  All threads of the CTA call it.
template <int NT, class VAt>
__device__ void accumulate_q1(VAt vat, int r, double2* Q, double* se, double* stau, double2* salpha, double2* sph,
                              double2* part) {
  const int tid = threadIdx.x;
  // Q1 = P_0 P_1 ... P_{r-3} (in Q), backward accumulation on the trailing block
  for (int idx = tid; idx < r * r; idx += NT) {
    const int i = idx / r, j = idx - (idx / r) * r;
    Q[idx] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = r - 3; k >= 0; --k) {
    const double tau = stau[k];
    if (tau == 0.0) continue;
    const int m = r - k - 1;
    // u_j = sum_i conj(v_i) Q[k+1+i][k+1+j], then Q_sub -= tau v u; with fewer columns than
    // threads the i range is split into G slices summed separately, then in a fixed order
    const int G = m <= NT ? min(8, NT / m) : 1;
    if (G > 1) {
      for (int idx = tid; idx < m * G; idx += NT) {
        const int j = idx % m, g = idx / m;
        const int i1 = (g + 1) * m / G;
        double2 s = make_double2(0.0, 0.0);
        for (int i = g * m / G; i < i1; ++i) s = cmacc(s, vat(k, i), Q[(k + 1 + i) * r + (k + 1 + j)]);
        part[idx] = s;
      }
      __syncthreads();
      for (int j = tid; j < m; j += NT) {
        double2 s = part[j];
        for (int g = 1; g < G; ++g) s = make_double2(s.x + part[g * m + j].x, s.y + part[g * m + j].y);
        sph[j] = make_double2(tau * s.x, tau * s.y);
      }
    } else {
      for (int j = tid; j < m; j += NT) {
        double2 s = make_double2(0.0, 0.0);
        for (int i = 0; i < m; ++i) s = cmacc(s, vat(k, i), Q[(k + 1 + i) * r + (k + 1 + j)]);
        sph[j] = make_double2(tau * s.x, tau * s.y);
      }
    }
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += NT) {
      const int i = idx / m, j = idx - (idx / m) * m;
      const double2 v = vat(k, i), u = sph[j];
      double2 a = Q[(k + 1 + i) * r + (k + 1 + j)];
      a.x = fma(-v.x, u.x, fma(v.y, u.y, a.x));
      a.y = fma(-v.x, u.y, fma(-v.y, u.x, a.y));
      Q[(k + 1 + i) * r + (k + 1 + j)] = a;
    }
    __syncthreads();
  }

  // phases: D_0 = 1, D_{k+1} = D_k e_k / |e_k| makes D^H T D real with
  // off-diagonal |e_k|; Z = Q1 D
  if (tid == 0) {
    double2 D = make_double2(1.0, 0.0);
    sph[0] = D;
    for (int k = 0; k + 1 < r; ++k) {
      const double2 e = salpha[k];
      const double ae = hypot(e.x, e.y);
      se[k] = ae;
      if (ae > 0.0) {
        const double2 u = make_double2(e.x / ae, e.y / ae);
        D = make_double2(D.x * u.x - D.y * u.y, D.x * u.y + D.y * u.x);
      }
      sph[k + 1] = D;
    }
    se[r - 1] = 0.0;
  }
  __syncthreads();
  for (int idx = tid; idx < r * r; idx += NT) {
    const int j = idx - (idx / r) * r;
    const double2 a = Q[idx], D = sph[j];
    Q[idx] = make_double2(a.x * D.x - a.y * D.y, a.x * D.y + a.y * D.x);
  }
  __syncthreads();
}

// Householder tridiagonalisation of the Hermitian r x r matrix H (row-major, full storage;
// overwritten, the Householder vectors end up below its subdiagonal).  For column k,
// x = H[k+1:, k], alpha = -phase(x_0) ||x||, v = x - alpha e_1, tau = 1 / (||x|| (||x|| + |x_0|)),
// P = I - tau v v^H, and H_sub <- P H_sub P = H_sub - v w^H - w v^H with p = tau H_sub v,
// w = p - (tau/2)(v^H p) v.  Then Q1 = P_0 ... P_{r-3} (backward accumulation) and the
// phases D_0 = 1, D_{k+1} = D_k e_k / |e_k|, which make D^H T D real with off-diagonal
// |e_k|.  Output: Q = Q1 D (r x r row-major), sd = diagonal of T, se = |e| (se[r-1] = 0).
// Scratch: stau, salpha, sph (shared, r entries each), pv (r entries, any memory; may
// alias Q's first row), red (NT/32 doubles), part (shared, NT entries).  All threads of the CTA
// call it.
template <int NT>
__device__ void herm_tridiag(double2* H, int r, double2* Q, double* sd, double* se, double* stau, double2* salpha,
                             double2* sph, double2* pv, double* red, double2* part) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k + 2 < r; ++k) {
    const int m = r - k - 1;
    double nx2 = 0.0;
    for (int i = tid; i < m; i += NT) {
      const double2 x = H[(k + 1 + i) * r + k];
      nx2 += x.x * x.x + x.y * x.y;
    }
    nx2 = blk_sum<NT>(nx2, red);
    if (tid == 0) sd[k] = H[k * r + k].x;
    if (!(nx2 > 0.0)) {  // column already reduced
      if (tid == 0) {
        stau[k] = 0.0;
        salpha[k] = make_double2(0.0, 0.0);
      }
      continue;
    }
    const double nx = sqrt(nx2);
    const double2 x0 = H[(k + 1) * r + k];
    const double a0 = hypot(x0.x, x0.y);
    const double2 ph = a0 > 0.0 ? make_double2(x0.x / a0, x0.y / a0) : make_double2(1.0, 0.0);
    const double tau = 1.0 / (nx * (nx + a0));
    // v_0 = x_0 - alpha = ph (|x_0| + ||x||); the other entries of v are those of x
    __syncthreads();  // every thread has read x_0 before it is overwritten
    if (tid == 0) {
      H[(k + 1) * r + k] = make_double2(ph.x * (a0 + nx), ph.y * (a0 + nx));
      stau[k] = tau;
      salpha[k] = make_double2(-ph.x * nx, -ph.y * nx);
    }
    __syncthreads();
    // p = tau H_sub v: one warp per row, lanes along the row
    for (int i = warp; i < m; i += NT / 32) {
      double2 s = make_double2(0.0, 0.0);
      const double2* hrow = H + (size_t)(k + 1 + i) * r + (k + 1);
      for (int j = lane; j < m; j += 32) s = cmac(s, hrow[j], H[(k + 1 + j) * r + k]);
      for (int off = 16; off > 0; off >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
      }
      if (lane == 0) pv[i] = make_double2(tau * s.x, tau * s.y);
    }
    __syncthreads();
    // K = (tau/2) v^H p (real for Hermitian H_sub)
    double kr = 0.0;
    for (int i = tid; i < m; i += NT) {
      const double2 v = H[(k + 1 + i) * r + k], p = pv[i];
      kr += fma(v.x, p.x, v.y * p.y);
    }
    kr = 0.5 * tau * blk_sum<NT>(kr, red);
    // w = p - K v (in place of p)
    for (int i = tid; i < m; i += NT) {
      const double2 v = H[(k + 1 + i) * r + k], p = pv[i];
      pv[i] = make_double2(fma(-kr, v.x, p.x), fma(-kr, v.y, p.y));
    }
    __syncthreads();
    // H_sub -= v w^H + w v^H on the lower triangle, mirrored into the upper one
    for (int e = tid; e < m * (m + 1) / 2; e += NT) {
      int i, j;
      tri_rc(e, i, j);
      const double2 vi = H[(k + 1 + i) * r + k], vj = H[(k + 1 + j) * r + k];
      const double2 wi = pv[i], wj = pv[j];
      double2 a = H[(k + 1 + i) * r + (k + 1 + j)];
      // a - vi conj(wj) - wi conj(vj)
      a.x = fma(-vi.x, wj.x, fma(-vi.y, wj.y, fma(-wi.x, vj.x, fma(-wi.y, vj.y, a.x))));
      a.y = fma(-vi.y, wj.x, fma(vi.x, wj.y, fma(-wi.y, vj.x, fma(wi.x, vj.y, a.y))));
      if (i == j) a.y = 0.0;
      H[(k + 1 + i) * r + (k + 1 + j)] = a;
      if (i != j) H[(k + 1 + j) * r + (k + 1 + i)] = make_double2(a.x, -a.y);
    }
    __syncthreads();
  }
  // the last 2 x 2 block is already tridiagonal
  if (tid == 0) {
    for (int k = (r >= 2 ? r - 2 : 0); k < r; ++k) sd[k] = H[k * r + k].x;
    if (r >= 2) {
      salpha[r - 2] = H[(r - 1) * r + (r - 2)];
      stau[r - 2] = 0.0;
    }
  }
  __syncthreads();

  accumulate_q1<NT>([&](int k, int i) { return H[(k + 1 + i) * r + k]; }, r, Q, se, stau, salpha, sph, part);
}

// Offset of entry (a, b), b <= a, in a packed lower triangle (row a holds columns 0..a).
__device__ __forceinline__ int tri_at(int a, int b) { return a * (a + 1) / 2 + b; }

// herm_tridiag for a matrix held in shared memory as its packed lower triangle H (tri_at), with
// the same reflectors, outputs and conventions (Q = Q1 D row-major in any memory, sd, se, stau,
// salpha; the Householder vectors end up below the subdiagonal of H's columns).  Per column
// five CTA barriers: (B) the reflector's vector v, (C) p = tau H_sub v as partial sums of column
// blocks (one item per row and block, no warp reductions on the FP64 pipe), (D) the totals per
// row and the real part of v^H p, (E) w = p - K v, (A) the rank-2 update of the lower triangle,
// which also sums the squares of the next column.  Scratch (shared): sv, sp (r entries each),
// red, red2 (NT/32 each), part (NT entries).  All threads of the CTA call it.
template <int NT>
__device__ void herm_tridiag_packed(double2* __restrict__ H, int r, double2* __restrict__ Q, double* sd, double* se,
                                    double* stau, double2* salpha, double2* __restrict__ sv,
                                    double2* __restrict__ sp, double* red, double* red2, double2* __restrict__ part) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {  // squares of the first column below the diagonal
    double q = 0.0;
    for (int i = 1 + tid; i < r; i += NT) {
      const double2 x = H[tri_at(i, 0)];
      q = fma(x.x, x.x, fma(x.y, x.y, q));
    }
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) red2[warp] = q;
  }
  __syncthreads();
  for (int k = 0; k + 2 < r; ++k) {
    const int m = r - k - 1, K = k + 1;
    double nx2 = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) nx2 += red2[w];
    if (tid == 0) sd[k] = H[tri_at(k, k)].x;
    if (!(nx2 > 0.0)) {  // column already reduced: no reflector; the next column's squares
      if (tid == 0) {
        stau[k] = 0.0;
        salpha[k] = make_double2(0.0, 0.0);
      }
      double q = 0.0;
      for (int i = 1 + tid; i < m; i += NT) {
        const double2 x = H[tri_at(K + i, K)];
        q = fma(x.x, x.x, fma(x.y, x.y, q));
      }
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      __syncthreads();  // every thread has read red2
      if (lane == 0) red2[warp] = q;
      __syncthreads();
      continue;
    }
    const double nx = sqrt(nx2);
    const double2 x0 = H[tri_at(K, k)];
    const double a0 = hypot(x0.x, x0.y);
    const double2 ph = a0 > 0.0 ? make_double2(x0.x / a0, x0.y / a0) : make_double2(1.0, 0.0);
    const double tau = 1.0 / (nx * (nx + a0));
    // v_0 = x_0 - alpha = ph (|x_0| + ||x||); the other entries of v are those of x
    const double2 v0 = make_double2(ph.x * (a0 + nx), ph.y * (a0 + nx));
    for (int i = tid; i < m; i += NT) sv[i] = i == 0 ? v0 : H[tri_at(K + i, k)];
    __syncthreads();  // (B) v complete; every thread has read x_0 and red2
    if (tid == 0) {   // nothing reads this entry again before the accumulation of Q1
      H[tri_at(K, k)] = v0;
      stau[k] = tau;
      salpha[k] = make_double2(-ph.x * nx, -ph.y * nx);
    }
    // p = tau H_sub v: item t = b m + i sums row i over the columns of block b (nb blocks of bw),
    // reading the upper part of a row as the conjugate of the stored column
    const int nb = min((m + 3) / 4, max(1, NT / m));
    const int bw = (m + nb - 1) / nb;
    for (int t = tid; t < m * nb; t += NT) {
      const int b = t / m, i = t - b * m;
      const int j1 = min(m, (b + 1) * bw);
      double2 acc = make_double2(0.0, 0.0);
      for (int j = b * bw; j < j1; ++j) {
        const bool lo = j <= i;
        double2 h = H[lo ? tri_at(K + i, K + j) : tri_at(K + j, K + i)];
        if (!lo) h.y = -h.y;
        acc = cmac(acc, h, sv[j]);
      }
      part[t] = acc;
    }
    __syncthreads();  // (C)
    double kp = 0.0;  // this thread's part of Re(v^H p)
    for (int i = tid; i < m; i += NT) {
      double2 q = part[i];
      for (int b = 1; b < nb; ++b) {
        const double2 u = part[b * m + i];
        q.x += u.x;
        q.y += u.y;
      }
      const double2 p = make_double2(tau * q.x, tau * q.y), v = sv[i];
      sp[i] = p;
      kp = fma(v.x, p.x, fma(v.y, p.y, kp));
    }
    if (warp * 32 < m)  // warps without rows contribute zero
      for (int o = 16; o > 0; o >>= 1) kp += __shfl_xor_sync(0xffffffffu, kp, o);
    if (lane == 0) red[warp] = kp;
    __syncthreads();  // (D)
    {  // w = p - K v in place of p, K = (tau/2) v^H p (real)
      double kr = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) kr += red[w];
      kr *= 0.5 * tau;
      for (int i = tid; i < m; i += NT) {
        const double2 v = sv[i], p = sp[i];
        sp[i] = make_double2(fma(-kr, v.x, p.x), fma(-kr, v.y, p.y));
      }
    }
    __syncthreads();  // (E)
    // H_sub -= v w^H + w v^H on the lower triangle.
    // Rows are taken in pairs (a, m - 1 - a), m + 1 entries per pair, so that a flat index maps
    // to (i, j) with one division; the middle row of an odd m is alone in its pair.
    const int len = m + 1, npair = (m + 1) / 2;
    const float rlen = 1.0f / (float)len;
    double q = 0.0;  // squares of the next column (j = 0, i >= 1)
    for (int e = tid; e < npair * len; e += NT) {
      int pr = (int)((float)e * rlen);
      if (pr * len > e) --pr;
      else if ((pr + 1) * len <= e) ++pr;
      const int c = e - pr * len;
      int i = pr, j = c;
      if (c > pr) {
        i = m - 1 - pr;
        j = c - pr - 1;
        if (i == pr) continue;
      }
      const double2 vi = sv[i], vj = sv[j], wi = sp[i], wj = sp[j];
      double2* h = H + tri_at(K + i, K + j);
      double2 a = *h;
      // a - vi conj(wj) - wi conj(vj)
      a.x = fma(-vi.x, wj.x, fma(-vi.y, wj.y, fma(-wi.x, vj.x, fma(-wi.y, vj.y, a.x))));
      a.y = fma(-vi.y, wj.x, fma(vi.x, wj.y, fma(-wi.y, vj.x, fma(wi.x, vj.y, a.y))));
      if (i == j) a.y = 0.0;
      *h = a;
      if (j == 0 && i >= 1) q = fma(a.x, a.x, fma(a.y, a.y, q));
    }
    if (__any_sync(0xffffffffu, q != 0.0))
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) red2[warp] = q;
    __syncthreads();  // (A)
  }
  // the last 2 x 2 block is already tridiagonal
  if (tid == 0) {
    for (int k = (r >= 2 ? r - 2 : 0); k < r; ++k) sd[k] = H[tri_at(k, k)].x;
    if (r >= 2) {
      salpha[r - 2] = H[tri_at(r - 1, r - 2)];
      stau[r - 2] = 0.0;
    }
  }
  __syncthreads();
  accumulate_q1<NT>([&](int k, int i) { return H[tri_at(k + 1 + i, k)]; }, r, Q, se, stau, salpha, sv, part);
}

// One Givens step of the implicit QL chase: from f = s e_i, g, returns c, s and h = |(f, g)|
// (h = 0 means the step underflowed).  rsqrt in the usual range, hypot outside it.
__device__ __forceinline__ void ql_givens(double f, double g, double& c, double& s, double& h) {
  const double h2 = fma(f, f, g * g);
  if (h2 > 1e-280 && h2 < 1e280) {
    const double rh = rsqrt(h2);
    h = h2 * rh;
    s = f * rh;
    c = g * rh;
  } else {
    h = hypot(f, g);
    s = h == 0.0 ? 0.0 : f / h;
    c = h == 0.0 ? 1.0 : g / h;
  }
}

// Deflation test of QL: e_m is negligible when it is below eps times the neighbouring diagonal
// entries (relative) or below eps ||T|| (absolute; a backward perturbation of the same order
// as the Householder reduction's, and what lets clusters of eigenvalues at the rounding level
// of ||T|| deflate).
__device__ __forceinline__ bool ql_split(double e, double d0, double d1, double tn) {
  const double a = fabs(e);
  return a <= DBL_EPSILON * (fabs(d0) + fabs(d1)) || a <= DBL_EPSILON * tn;
}

// Implicit QL with Wilkinson-type shifts on the real symmetric tridiagonal (sd, se): the
// published implicit QL method of Bowdler, Martin, Reinsch and Wilkinson (the tql2 procedure of
// the Handbook for Automatic Computation, Vol. II), whose bulge chase this follows.  se[i]
// coupling i and i+1 (shared arrays).  Thread 0 chases one bulge at a time and records its
// rotations in rc, rs (shared, r entries); then every thread applies them to the rows of Z
// (r x r complex, row-major; real and imaginary parts independently):
//   Z[:, i+1] <- s Z[:, i] + c Z[:, i+1],  Z[:, i] <- c Z[:, i] - s Z[:, i+1],  i = m-1, m-2, ...
// sd becomes the eigenvalues.  flags: 4 shared ints.  Returns false on every thread when an
// eigenvalue needs more than max_iter chases.  All threads of the CTA call it.
template <int NT>
__device__ bool ql_single(double* sd, double* se, int r, double2* Z, double* rc, double* rs, int* flags,
                          int max_iter) {
  const int tid = threadIdx.x;
  int l = 0, iter = 0;  // thread 0's state
  double tn = 0.0;      // max_i |d_i| + |e_i| (thread 0)
  if (tid == 0)
    for (int i = 0; i < r; ++i) tn = fmax(tn, fabs(sd[i]) + fabs(se[i]));
  for (;;) {
    if (tid == 0) {
      flags[0] = 0;  // rotations of this sweep
      flags[2] = 0;  // done
      bool emitted = false;
      while (!emitted) {
        if (l >= r) {
          flags[2] = 1;
          break;
        }
        int m = l;
        while (m < r - 1 && !ql_split(se[m], sd[m], sd[m + 1], tn)) ++m;
        if (m == l) {
          ++l;
          iter = 0;
          continue;
        }
        if (++iter > max_iter) {
          flags[3] = 1;
          flags[2] = 1;
          break;
        }
        double g = (sd[l + 1] - sd[l]) / (2.0 * se[l]);
        double h = fabs(g) < 1e150 ? sqrt(fma(g, g, 1.0)) : fabs(g);
        g = sd[m] - sd[l] + se[l] / (g + (g >= 0.0 ? h : -h));
        double sn = 1.0, cs = 1.0, p = 0.0;
        int nrot = 0;
        bool underflow = false;
        for (int i = m - 1; i >= l; --i) {
          const double f = sn * se[i], b = cs * se[i];
          ql_givens(f, g, cs, sn, h);
          se[i + 1] = h;
          if (h == 0.0) {
            sd[i + 1] -= p;
            se[m] = 0.0;
            underflow = true;
            break;
          }
          g = sd[i + 1] - p;
          h = fma(sd[i] - g, sn, 2.0 * cs * b);
          p = sn * h;
          sd[i + 1] = g + p;
          g = fma(cs, h, -b);
          rc[nrot] = cs;
          rs[nrot] = sn;
          ++nrot;
        }
        if (!underflow) {
          sd[l] -= p;
          se[l] = g;
          se[m] = 0.0;
        }
        flags[0] = nrot;
        flags[1] = m;
        emitted = nrot > 0;
      }
    }
    __syncthreads();
    if (flags[2]) break;
    const int nrot = flags[0], m = flags[1];
    double* Zr = reinterpret_cast<double*>(Z);
    for (int rp = tid; rp < 2 * r; rp += NT) {
      const int row = rp >> 1, part = rp & 1;
      double* zrow = Zr + (size_t)2 * row * r + part;
      double hi = zrow[2 * m];
      for (int q = 0; q < nrot; ++q) {
        const int i = m - 1 - q;
        const double lo = zrow[2 * i];
        const double c = rc[q], s = rs[q];
        zrow[2 * (i + 1)] = fma(s, lo, c * hi);
        hi = fma(c, lo, -s * hi);
      }
      zrow[2 * (m - nrot)] = hi;
    }
    __syncthreads();
  }
  const bool ok = flags[3] == 0;
  __syncthreads();
  return ok;
}

}  // namespace hq
}  // namespace mrom
