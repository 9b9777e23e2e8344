// Off-line stage on the GPU: snapshot TSVD and Galerkin projection (Sects. 4.1-4.3).
//
//   G_D = D^H D                                  tall Gram (split over rows)
//   G_D = V Lambda V^H                           Householder tridiagonalisation + implicit QL (one CTA)
//   s_k = sqrt(lambda_k), r = #{s_k / s_1 >= TOL_Sigma} (capped)     (Eq. (15))
//   U   = D V_r diag(1/s_r)                      left singular vectors (Eq. (14))
//   Y   = K U                                    CSR SpMM
//   K_r = U^H Y, C_r = U^H diag(c) U, Me = U^H diag(eps m) U,
//   b_i = U^H (c o_i), c00 = o^T diag(c) o                             (Eqs. (17)-(19))
//   G   = Phi^H diag(1/x) Phi, Phi = [c o_i | Y + eps m U | c U]      (Lemma 4.2)
// Everything is float64 / complex128, except that the mixed projection mode forms the basis U
// (without a certificate, which needs U in float64), K U and the products K_r, C_r, eps M_r and b
// in complex64 (the snapshot Gram of the TSVD and the certificate Gram stay float64: TOL_Sigma
// down to 1e-6 needs the Gram's eigenvalues to 1e-12 of the largest).
// The float64 kernels are FP64-pipe bound on GB300
// (the snapshot and basis streams are re-read from L2), so they are written for
// full FP64 utilisation with register tiles rather than for HBM streaming.
#include "mrom_internal.h"
#include "herm_tridiag.cuh"
#include "tridiag_dc.cuh"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace mrom {
namespace {

__device__ __forceinline__ double2 c_conj_mac(double2 c, double2 a, double2 b) {  // c + conj(a) b
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}

// ------------------------------------------------------------------ tall Gram
// part[split][a][b] = sum_{n in split} conj(A[n][a]) * wgt(n) * B[n][b]
// Element (n, c) of A is A[n * rsA + c * csA] (any layout).  One CTA computes a Ta x Tb
// output tile (even sizes up to kGT, chosen so that the tiles cover ma x mb with little
// padding) over its row range; (Ta/2) (Tb/2) threads hold 2 x 2 outputs each.
constexpr int kGT = 32;
constexpr int kGR = 32;

// The 2 x 2 output block (ty, tx) of thread tid.  On a diagonal tile of a Hermitian product
// only the blocks with ty <= tx are computed (the rest is mirrored by the reduction), with
// the threads packed so that the idle ones form whole warps.
__device__ __forceinline__ void gram_thread_block(bool upper_only, int ha, int hb, int tid, bool& active, int& ty,
                                                  int& tx) {
  if (upper_only) {
    const int nu = hb * (hb + 1) / 2;
    active = tid < nu;
    int i = 0, j = 0;
    if (active) hq::tri_rc(nu - 1 - tid, i, j);  // i >= j in the reversed triangle
    ty = hb - 1 - i;
    tx = hb - 1 - j;
  } else {
    active = tid < ha * hb;
    ty = tid / hb;
    tx = tid - (tid / hb) * hb;
  }
}

__global__ void __launch_bounds__(256)
gram_partial_kernel(const double2* __restrict__ A, int64_t rsA, int64_t csA, int ma,
                    const double2* __restrict__ B, int64_t rsB, int64_t csB, int mb,
                    const double* __restrict__ w, int wmode, int64_t n, int64_t rows_per_split,
                    const int2* __restrict__ tiles, int Ta, int Tb, int herm, double2* __restrict__ part) {
  __shared__ double2 As[kGR][kGT + 1];
  __shared__ double2 Bs[kGR][kGT + 1];
  const int tid = threadIdx.x;
  const int hb = Tb >> 1;
  const int2 tile = tiles[blockIdx.y];
  bool active;
  int ty, tx;
  gram_thread_block(herm && tile.x == tile.y, Ta >> 1, hb, tid, active, ty, tx);
  const int a_base = tile.x * Ta, b_base = tile.y * Tb;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_split;
  const int64_t r1 = min(n, r0 + rows_per_split);
  double2 acc[2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
  for (int64_t row0 = r0; row0 < r1; row0 += kGR) {
    for (int idx = tid; idx < kGR * Ta; idx += 256) {
      int rr, cc;
      if (csA == 1) { rr = idx / Ta; cc = idx - rr * Ta; } else { cc = idx / kGR; rr = idx - cc * kGR; }
      const int64_t nr = row0 + rr;
      const int col = a_base + cc;
      As[rr][cc] = (nr < r1 && col < ma) ? A[nr * rsA + col * csA] : make_double2(0.0, 0.0);
    }
    for (int idx = tid; idx < kGR * Tb; idx += 256) {
      int rr, cc;
      if (csB == 1) { rr = idx / Tb; cc = idx - rr * Tb; } else { cc = idx / kGR; rr = idx - cc * kGR; }
      const int64_t nb = row0 + rr;
      const int colb = b_base + cc;
      double2 v = make_double2(0.0, 0.0);
      if (nb < r1 && colb < mb) {
        v = B[nb * rsB + colb * csB];
        if (wmode) {
          const double s = (wmode == 1) ? w[nb] : 1.0 / w[nb];
          v.x *= s;
          v.y *= s;
        }
      }
      Bs[rr][cc] = v;
    }
    __syncthreads();
    if (active) {
#pragma unroll 8
      for (int rr = 0; rr < kGR; ++rr) {
        const double2 a0 = As[rr][ty * 2], a1 = As[rr][ty * 2 + 1];
        const double2 b0 = Bs[rr][tx * 2], b1 = Bs[rr][tx * 2 + 1];
        acc[0][0] = c_conj_mac(acc[0][0], a0, b0);
        acc[0][1] = c_conj_mac(acc[0][1], a0, b1);
        acc[1][0] = c_conj_mac(acc[1][0], a1, b0);
        acc[1][1] = c_conj_mac(acc[1][1], a1, b1);
      }
    }
    __syncthreads();
  }
  if (!active) return;
  double2* out = part + (size_t)blockIdx.x * ma * mb;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int a = a_base + ty * 2 + i, b = b_base + tx * 2 + j;
      if (a < ma && b < mb) out[(size_t)a * mb + b] = acc[i][j];
    }
}

// Gram of at most 4 x 4 columns (e.g. c00 = O^T C O): per thread a register block over a
// grid-stride range of rows, then a fixed-order reduction over the CTA into part[block][ma x mb].
constexpr int kGS = 4;
__global__ void __launch_bounds__(256)
gram_small_kernel(const double2* __restrict__ A, int64_t rsA, int64_t csA, int ma, const double2* __restrict__ B,
                  int64_t rsB, int64_t csB, int mb, const double* __restrict__ w, int wmode, int64_t n,
                  double2* __restrict__ part) {
  __shared__ double2 red[8][kGS * kGS];
  double2 acc[kGS][kGS];
#pragma unroll
  for (int i = 0; i < kGS; ++i)
#pragma unroll
    for (int j = 0; j < kGS; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int64_t row = (int64_t)blockIdx.x * 256 + threadIdx.x; row < n; row += (int64_t)gridDim.x * 256) {
    double2 a[kGS], b[kGS];
    const double s = wmode == 0 ? 1.0 : (wmode == 1 ? w[row] : 1.0 / w[row]);
#pragma unroll
    for (int i = 0; i < kGS; ++i) {
      a[i] = i < ma ? A[row * rsA + i * csA] : make_double2(0.0, 0.0);
      const double2 v = i < mb ? B[row * rsB + i * csB] : make_double2(0.0, 0.0);
      b[i] = make_double2(s * v.x, s * v.y);
    }
#pragma unroll
    for (int i = 0; i < kGS; ++i)
#pragma unroll
      for (int j = 0; j < kGS; ++j) acc[i][j] = c_conj_mac(acc[i][j], a[i], b[j]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kGS; ++i)
#pragma unroll
    for (int j = 0; j < kGS; ++j) {
      double2 v = acc[i][j];
      for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      }
      if (lane == 0) red[warp][i * kGS + j] = v;
    }
  __syncthreads();
  if (threadIdx.x < ma * mb) {
    const int i = threadIdx.x / mb, j = threadIdx.x - (threadIdx.x / mb) * mb;
    double2 v = make_double2(0.0, 0.0);
    for (int k = 0; k < 8; ++k) v = make_double2(v.x + red[k][i * kGS + j].x, v.y + red[k][i * kGS + j].y);
    part[(size_t)blockIdx.x * ma * mb + threadIdx.x] = v;
  }
}

__global__ void __launch_bounds__(256)
spmm_csr_f32_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                    const float* __restrict__ val, int64_t n, const float2* __restrict__ U, int r,
                    float2* __restrict__ Y) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float2 acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (int k = rowptr[row]; k < rowptr[row + 1]; ++k) {
    const int64_t j = col[k];
    const float v = val[k];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lane + 32 * q;
      if (c < r) {
        const float2 u = U[j * r + c];
        acc[q].x = fmaf(v, u.x, acc[q].x);
        acc[q].y = fmaf(v, u.y, acc[q].y);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = lane + 32 * q;
    if (c < r) Y[row * r + c] = acc[q];
  }
}

__global__ void to_f32_kernel(const double* __restrict__ x, int64_t n, double scale, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)(scale * x[i]);
}

// G[a][b] = sum over splits (fixed order).  Hermitian: the upper triangle was computed
// (tiles with b-tile >= a-tile, upper blocks of the diagonal tiles); the rest is mirrored
// and the diagonal made real.
__global__ void gram_reduce_kernel(const double2* __restrict__ part, int nsplit, int ma, int mb, int hermitian,
                                   int T, double2* __restrict__ G, int64_t ldg) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)ma * mb;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / mb), b = (int)(idx % mb);
    int sa = a, sb = b;
    bool conj = false;
    if (hermitian && b < a) {
      sa = b;
      sb = a;
      conj = true;
    }
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < nsplit; ++k) {
      const double2 v = part[(size_t)k * ma * mb + (size_t)sa * mb + sb];
      s.x += v.x;
      s.y += v.y;
    }
    if (conj) s.y = -s.y;
    if (hermitian && a == b) s.y = 0.0;
    G[(int64_t)a * ldg + b] = s;
  }
}

// ------------------------------------------------ Householder + tridiagonal eigensolver
// Hermitian m x m A = Z Lambda Z^H (A overwritten): Householder tridiagonalisation, then the real
// tridiagonal by divide and conquer (m <= MROM_MAX_R, with `work`: 3 m^2 float64) and Z = Q1 D Z2,
// or else implicit QL with the rotations accumulated into Z (columns = eigenvectors).  One CTA.
// *status gets kStatusTimeout if QL did not converge or divide and conquer met a non-finite value.
constexpr int kEigThreads = 512;

// One CTA per matrix: CTA b takes A + b m^2, Z + b m^2, lam + b m (and work + 3 b m^2).
__global__ void __launch_bounds__(kEigThreads)
herm_eig_kernel(double2* __restrict__ A, int m, double2* __restrict__ Z, double* __restrict__ lam,
                int* __restrict__ status, double* __restrict__ work) {
  A += (size_t)blockIdx.x * m * m;
  Z += (size_t)blockIdx.x * m * m;
  lam += (size_t)blockIdx.x * m;
  if (work) work += (size_t)blockIdx.x * 3 * m * m;
  __shared__ double sd[MROM_MAX_SNAPSHOTS], se[MROM_MAX_SNAPSHOTS], stau[MROM_MAX_SNAPSHOTS];
  __shared__ double rc[MROM_MAX_SNAPSHOTS], rs[MROM_MAX_SNAPSHOTS];
  __shared__ double2 salpha[MROM_MAX_SNAPSHOTS], sph[MROM_MAX_SNAPSHOTS], pv[MROM_MAX_SNAPSHOTS];
  __shared__ double red[kEigThreads / 32];
  __shared__ double2 part[kEigThreads];
  __shared__ int flags[4];
  if (threadIdx.x < 4) flags[threadIdx.x] = 0;
  __syncthreads();
  hq::herm_tridiag<kEigThreads>(A, m, Z, sd, se, stau, salpha, sph, pv, red, part);
  if (work != nullptr && m <= dc::kDcMaxN) {
    __shared__ dc::DcShared S;
    const int mm = m * m;
    const double* Z2 = dc::tridiag_dc<kEigThreads>(sd, se, m, work, work + mm, work + 2 * mm, S);
    // Z Z2 into A (the Householder vectors are no longer needed), then back into Z
    for (int idx = threadIdx.x; idx < mm; idx += kEigThreads) {
      const int i = idx / m, j = idx - (idx / m) * m;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < m; ++k) {
        const double2 zk = Z[i * m + k];
        const double q = Z2[k * m + j];
        acc.x = fma(zk.x, q, acc.x);
        acc.y = fma(zk.y, q, acc.y);
      }
      A[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < mm; idx += kEigThreads) Z[idx] = A[idx];
    for (int i = threadIdx.x; i < m; i += kEigThreads) lam[i] = S.lam[i];
    if (threadIdx.x == 0 && S.bad) atomicOr(status, kStatusTimeout);
    return;
  }
  const bool ok = hq::ql_single<kEigThreads>(sd, se, m, Z, rc, rs, flags, 60);
  for (int i = threadIdx.x; i < m; i += kEigThreads) lam[i] = sd[i];
  if (threadIdx.x == 0 && !ok) atomicOr(status, kStatusTimeout);
}

// ------------------------------------------------------------- basis apply
// U[row][off + k] = sum_c D(row, c) W[c][k] for k < r; D(row, c) = D[c * ldd + row] (complex128
// columns), W (m x r, row-major) in shared memory, U row-major (ldu).  One thread per row, 16
// output columns per pass with the accumulators in registers; each pass is staged in shared
// memory and written row segment by row segment (coalesced).  T = double2 (float64, the float64
// projection) or float2 (the mixed projection's complex64 basis, float32 accumulation over the
// m snapshot columns).
constexpr int kAR = 128;  // rows per CTA (one per thread)
constexpr int kAC = 16;   // output columns per pass

template <class T>
__device__ __forceinline__ T cplx_mac(T c, T a, T b) {  // c + a b
  c.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
  c.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
  return c;
}

template <class T>
__global__ void __launch_bounds__(kAR)
apply_basis_kernel(const double2* __restrict__ D, int64_t ldd, int m, int64_t n, const T* __restrict__ W, int r,
                   T* __restrict__ U, int64_t ldu) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Wt = reinterpret_cast<T*>(smem_raw);  // m x kAC: the pass's columns of W
  T* St = Wt + (size_t)m * kAC;            // kAR x (kAC + 1): the pass's outputs
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * kAR, row = row0 + tid;
  for (int k0 = 0; k0 < r; k0 += kAC) {
    const int kc = min(kAC, r - k0);
    __syncthreads();  // the previous pass's stage written out
    for (int idx = tid; idx < m * kAC; idx += kAR) {
      const int c = idx / kAC, k = idx - (idx / kAC) * kAC;
      T w;
      w.x = w.y = 0;
      if (k < kc) w = W[(size_t)c * r + k0 + k];
      Wt[idx] = w;
    }
    __syncthreads();
    T acc[kAC];
#pragma unroll
    for (int k = 0; k < kAC; ++k) acc[k].x = acc[k].y = 0;
    if (row < n) {
      for (int c = 0; c < m; ++c) {
        const double2 d64 = D[(int64_t)c * ldd + row];
        T d;
        d.x = d64.x;
        d.y = d64.y;
        const T* w = Wt + (size_t)c * kAC;
#pragma unroll
        for (int k = 0; k < kAC; ++k) acc[k] = cplx_mac(acc[k], d, w[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < kAC; ++k) St[tid * (kAC + 1) + k] = acc[k];
    __syncthreads();
    for (int idx = tid; idx < kAR * kc; idx += kAR) {
      const int rr = idx / kc, k = idx - (idx / kc) * kc;
      if (row0 + rr < n) U[(row0 + rr) * ldu + k0 + k] = St[rr * (kAC + 1) + k];
    }
  }
}

// ------------------------------------------------------------------- SpMM
// Y[row][:] = sum_k K_val[k] U[K_col[k]][:] (+ e[row] U[row][:]); one warp per row.
__global__ void __launch_bounds__(256)
spmm_csr_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                const double* __restrict__ val, int64_t n, const double2* __restrict__ U, int r,
                const double* __restrict__ e, double2* __restrict__ Y) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double2 acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (int k = rowptr[row]; k < rowptr[row + 1]; ++k) {
    const int64_t j = col[k];
    const double v = val[k];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lane + 32 * q;
      if (c < r) {
        const double2 u = U[j * r + c];
        acc[q].x = fma(v, u.x, acc[q].x);
        acc[q].y = fma(v, u.y, acc[q].y);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = lane + 32 * q;
    if (c < r) {
      double2 y = acc[q];
      if (e) {
        const double2 u = U[row * r + c];
        y.x = fma(e[row], u.x, y.x);
        y.y = fma(e[row], u.y, y.y);
      }
      Y[row * r + c] = y;
    }
  }
}

// Oc[row][i] = o[i][row] + 0i (3 directions)
__global__ void complexify_o_kernel(const double* __restrict__ o, int64_t n, double2* __restrict__ Oc) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 3 * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / 3;
    const int i = (int)(idx % 3);
    Oc[idx] = make_double2(o[(int64_t)i * n + row], 0.0);
  }
}

// Phi[row] = [c o_1, c o_2, c o_3 | Y + eps m U | c U]  (width 2r + 3)
__global__ void build_phi_kernel(const double* __restrict__ o, const double* __restrict__ cdiag,
                                 const double* __restrict__ mdiag, double eps, const double2* __restrict__ Y,
                                 const double2* __restrict__ U, int r, int64_t n, double2* __restrict__ Phi) {
  const int wdt = 2 * r + 3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)wdt * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / wdt;
    const int k = (int)(idx % wdt);
    const double c = cdiag[row];
    double2 v;
    if (k < 3) {
      v = make_double2(c * o[(int64_t)k * n + row], 0.0);
    } else if (k < 3 + r) {
      const double2 y = Y[row * r + (k - 3)];
      const double2 u = U[row * r + (k - 3)];
      const double em = mdiag ? eps * mdiag[row] : 0.0;
      v = make_double2(fma(em, u.x, y.x), fma(em, u.y, y.y));
    } else {
      const double2 u = U[row * r + (k - 3 - r)];
      v = make_double2(c * u.x, c * u.y);
    }
    Phi[idx] = v;
  }
}

// Y[c * n + i] = X[c * ldx + i] + 0i for n_c columns
__global__ void real_cols_kernel(const double* __restrict__ X, int64_t ldx, int64_t n, int n_c,
                                 double2* __restrict__ Y) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * n_c;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / n, i = idx - (idx / n) * n;
    Y[idx] = make_double2(X[c * ldx + i], 0.0);
  }
}

// Phi_ext[row] = [c x_1..3 | c V | (K U - K_in U) + eps m U | K_in U | c U]  (width 3 + m + 3 r):
// the residual basis of the certificate at a permeability scale
__global__ void build_phi_ext_kernel(const double2* __restrict__ X3, const double2* __restrict__ V, int m,
                                     const double2* __restrict__ U, const double2* __restrict__ KU,
                                     const double2* __restrict__ KinU, int r, const double* __restrict__ cdiag,
                                     const double* __restrict__ mdiag, double eps, int64_t n,
                                     double2* __restrict__ Phi) {
  const int w = 3 + m + 3 * r;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * w;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / w;
    const int col = (int)(idx - row * w);
    const double c = cdiag[row];
    double2 v;
    if (col < 3) {
      const double2 x = X3[row * 3 + col];
      v = make_double2(c * x.x, c * x.y);
    } else if (col < 3 + m) {
      const double2 x = V[row * m + col - 3];
      v = make_double2(c * x.x, c * x.y);
    } else if (col < 3 + m + r) {
      const int k = col - 3 - m;
      const double2 a = KU[row * r + k], b = KinU[row * r + k], u = U[row * r + k];
      const double em = mdiag ? eps * mdiag[row] : 0.0;
      v = make_double2(a.x - b.x + em * u.x, a.y - b.y + em * u.y);
    } else if (col < 3 + m + 2 * r) {
      v = KinU[row * r + col - 3 - m - r];
    } else {
      const double2 u = U[row * r + col - 3 - m - 2 * r];
      v = make_double2(c * u.x, c * u.y);
    }
    Phi[idx] = v;
  }
}

// Z = X - Y (n complex values)
__global__ void csub_kernel(const double2* __restrict__ X, const double2* __restrict__ Y, int n,
                            double2* __restrict__ Z) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x)
    Z[idx] = make_double2(X[idx].x - Y[idx].x, X[idx].y - Y[idx].y);
}

__global__ void scale_kernel(const double* __restrict__ x, double a, int64_t n, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

__global__ void recip_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = 1.0 / x[i];
}

// UO[n] = [U[n][0..r) | O[n][0..3)] (row-major, r + 3 columns)
__global__ void concat_uo_kernel(const double2* __restrict__ U, int r, const double2* __restrict__ O, int64_t n,
                                 double2* __restrict__ UO) {
  const int m = r + 3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / m;
    const int c = (int)(idx - row * m);
    UO[idx] = c < r ? U[row * r + c] : O[row * 3 + (c - r)];
  }
}

// Blocks of the (r+3) x (r+3) Gram of [U | O]: C_r (r x r), B = U^H C O (r x 3), c00 (3 x 3).
__global__ void split_uo_kernel(const double2* __restrict__ G, int r, double2* __restrict__ Cr,
                                double2* __restrict__ Bm, double2* __restrict__ c00) {
  const int m = r + 3;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * m; idx += gridDim.x * blockDim.x) {
    const int a = idx / m, b = idx - (idx / m) * m;
    const double2 v = G[idx];
    if (a < r && b < r) Cr[a * r + b] = v;
    else if (a < r) Bm[a * 3 + (b - r)] = v;
    else if (b >= r) c00[(a - r) * 3 + (b - r)] = v;
  }
}

__global__ void symmetrize_kernel(double2* __restrict__ G, int m) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * m; idx += gridDim.x * blockDim.x) {
    const int a = idx / m, b = idx % m;
    if (a > b) continue;
    const double2 x = G[a * m + b], y = G[b * m + a];
    const double2 s = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
    G[a * m + b] = s;
    G[b * m + a] = make_double2(s.x, -s.y);
    if (a == b) G[a * m + b].y = 0.0;
  }
}


}  // namespace

// Even tile size up to kGT that covers m with the fewest tiles and the least padding.
int gram_tile(int m) {
  const int nt = (m + kGT - 1) / kGT;
  const int t = 2 * ((m + 2 * nt - 1) / (2 * nt));
  return t < 2 ? 2 : t;
}

// G (ma x mb, row-major, ldg) = A^H diag(w) B over n rows; see gram_partial_kernel.
cudaError_t tall_gram(mrom_ctx* h, const double2* A, int64_t rsA, int64_t csA, int ma, const double2* B,
                      int64_t rsB, int64_t csB, int mb, const double* w, int wmode, int64_t n, bool hermitian,
                      double2* G, int64_t ldg) {
  if (ma <= kGS && mb <= kGS) {  // a few columns: one register block per thread
    const int64_t nb = std::max<int64_t>(1, std::min<int64_t>(4LL * h->num_sms, (n + 255) / 256));
    DevBuf part;
    cudaError_t e = cudaMalloc(&part.p, (size_t)nb * ma * mb * sizeof(double2));
    if (e != cudaSuccess) return e;
    gram_small_kernel<<<(unsigned)nb, 256, 0, h->stream>>>(A, rsA, csA, ma, B, rsB, csB, mb, w, wmode, n,
                                                          static_cast<double2*>(part.p));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gram_reduce_kernel<<<1, 256, 0, h->stream>>>(static_cast<double2*>(part.p), (int)nb, ma, mb, hermitian ? 1 : 0, 1,
                                                G, ldg);
    e = cudaGetLastError();
    h->launches += 2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // part is freed on return
    return e;
  }
  const int Ta = gram_tile(hermitian ? std::max(ma, mb) : ma), Tb = hermitian ? Ta : gram_tile(mb);
  const int ta = (ma + Ta - 1) / Ta, tb = (mb + Tb - 1) / Tb;
  std::vector<int2> tl;
  for (int i = 0; i < ta; ++i)
    for (int j = hermitian ? i : 0; j < tb; ++j) tl.push_back(make_int2(i, j));
  const int ntiles = (int)tl.size();
  // split the rows so that about 4 CTAs per SM run, each over at least 1024 rows
  int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>((4LL * h->num_sms + ntiles - 1) / ntiles,
                                                          (n + 1023) / 1024));
  nsplit = std::min<int64_t>(nsplit, 65535);
  const int64_t per = ((n + nsplit - 1) / nsplit + kGR - 1) / kGR * kGR;
  nsplit = (n + per - 1) / per;
  if (nsplit < 1) nsplit = 1;
  DevBuf part, tiles;
  cudaError_t e = cudaMalloc(&part.p, (size_t)nsplit * ma * mb * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&tiles.p, tl.size() * sizeof(int2));
  if (e == cudaSuccess) e = cudaMemcpyAsync(tiles.p, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)nsplit, (unsigned)ntiles);
  gram_partial_kernel<<<grid, 256, 0, h->stream>>>(A, rsA, csA, ma, B, rsB, csB, mb, w, wmode, n, per,
                                                  static_cast<int2*>(tiles.p), Ta, Tb, hermitian ? 1 : 0,
                                                  static_cast<double2*>(part.p));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int rb = (int)std::min<int64_t>(4096, ((int64_t)ma * mb + 255) / 256);
  gram_reduce_kernel<<<std::max(rb, 1), 256, 0, h->stream>>>(static_cast<double2*>(part.p), (int)nsplit, ma, mb,
                                                              hermitian ? 1 : 0, Ta, G, ldg);
  e = cudaGetLastError();
  h->launches += 2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // part/tiles are freed on return
  return e;
}

}  // namespace mrom

using namespace mrom;

namespace mrom {
namespace {

// Snapshot Gram, eigensolver and truncation for the m columns of D (column c at
// D + c * ldd): returns the rank r, the singular values (host) and W = V_r diag(1/s_r)
// (host, m x r, row-major) such that U = D W.
// Truncated SVD of nb snapshot sets of m columns each (set b at Dp + b * m * ldd): their Grams,
// one eigensolver launch with one CTA per set, then per set the singular values s[b], the rank
// r_out[b] (s_k / s_1 >= tol_sigma, at most r_cap) and W = V_r diag(1/s_r) in wh[b] (m x r).
mrom_status gram_eig_many(mrom_ctx* h, int nb, const double2* Dp, int64_t ldd, int64_t n, int m, double tol_sigma,
                          int r_cap, int* r_out, std::vector<double>* s, std::vector<double2>* wh) {
  cudaStream_t st = h->stream;
  const size_t mm = (size_t)m * m;
  DevBuf g, vbuf, lam, work;
  cudaError_t e = cudaMalloc(&g.p, nb * mm * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&vbuf.p, nb * mm * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&lam.p, nb * (size_t)m * sizeof(double));
  if (e == cudaSuccess && m <= dc::kDcMaxN) e = cudaMalloc(&work.p, 3 * nb * mm * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: allocation");
  for (int b = 0; b < nb && e == cudaSuccess; ++b) {
    const double2* D = Dp + (size_t)b * m * ldd;
    e = tall_gram(h, D, 1, ldd, m, D, 1, ldd, m, nullptr, 0, n, true, static_cast<double2*>(g.p) + b * mm, m);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: snapshot Gram");
  herm_eig_kernel<<<nb, kEigThreads, 0, st>>>(static_cast<double2*>(g.p), m, static_cast<double2*>(vbuf.p),
                                              static_cast<double*>(lam.p), h->d_status,
                                              static_cast<double*>(work.p));
  ++h->launches;
  std::vector<double> lh_all(nb * (size_t)m);
  std::vector<double2> vh_all(nb * mm);
  e = cudaMemcpyAsync(lh_all.data(), lam.p, lh_all.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(vh_all.data(), vbuf.p, vh_all.size() * sizeof(double2), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: eigensolver");
  int stw = 0;
  cudaMemcpy(&stw, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (stw & kStatusTimeout) {
    cudaMemset(h->d_status, 0, sizeof(int));
    return fail(h, MROM_ENOTCONVERGED, "mrom_project: the snapshot eigensolver did not converge (or met a non-finite value)");
  }
  for (int b = 0; b < nb; ++b) {
    const double* lh = lh_all.data() + (size_t)b * m;
    const double2* vh = vh_all.data() + b * mm;
    std::vector<int> order(m);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return lh[x] > lh[y]; });
    std::vector<double>& sb = s[b];
    sb.assign(m, 0.0);
    for (int k = 0; k < m; ++k) sb[k] = std::sqrt(std::max(lh[order[k]], 0.0));
    // truncation rule (Eq. (15) reading): keep s_k / s_1 >= TOL_Sigma, at most r_cap
    int r = 0;
    for (int k = 0; k < m; ++k)
      if (sb[0] > 0 && sb[k] > 0 && sb[k] / sb[0] >= tol_sigma) r = k + 1;
    r = std::min(r, r_cap);
    if (r < 1) return fail(h, MROM_EINVAL, "mrom_project: snapshots have no nonzero singular value");
    wh[b].assign((size_t)m * r, make_double2(0.0, 0.0));
    for (int c = 0; c < m; ++c)
      for (int k = 0; k < r; ++k) {
        const double2 v = vh[(size_t)c * m + order[k]];
        wh[b][(size_t)c * r + k] = make_double2(v.x / sb[k], v.y / sb[k]);
      }
    r_out[b] = r;
  }
  return MROM_OK;
}

mrom_status gram_eig(mrom_ctx* h, const double2* Dp, int64_t ldd, int64_t n, int m, double tol_sigma, int r_cap,
                     int* r_out, std::vector<double>& s, std::vector<double2>& wh) {
  return gram_eig_many(h, 1, Dp, ldd, n, m, tol_sigma, r_cap, r_out, &s, &wh);
}

// U[:, off : off + r] (row-major, leading dimension ldu) = D W, in float64 (U64) or complex64 (U32)
mrom_status apply_basis(mrom_ctx* h, const double2* Dp, int64_t ldd, int64_t n, int m, const std::vector<double2>& wh,
                        int r, double2* U64, int ldu, float2* U32 = nullptr) {
  DevBuf wbuf;
  const bool f32 = U32 != nullptr;
  const size_t esz = f32 ? sizeof(float2) : sizeof(double2);
  std::vector<float2> w32;
  if (f32) {
    w32.resize(wh.size());
    for (size_t k = 0; k < wh.size(); ++k) w32[k] = make_float2((float)wh[k].x, (float)wh[k].y);
  }
  const size_t smem = ((size_t)m * kAC + (size_t)kAR * (kAC + 1)) * esz;
  if (smem > h->smem_optin) return fail(h, MROM_EINVAL, "mrom_project: snapshot count too large for the basis apply");
  cudaError_t e = cudaMalloc(&wbuf.p, wh.size() * esz);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(wbuf.p, f32 ? static_cast<const void*>(w32.data()) : static_cast<const void*>(wh.data()),
                        wh.size() * esz, cudaMemcpyHostToDevice, h->stream);
  const unsigned grid = (unsigned)((n + kAR - 1) / kAR);
  if (f32) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(apply_basis_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      apply_basis_kernel<float2><<<grid, kAR, smem, h->stream>>>(Dp, ldd, m, n, static_cast<float2*>(wbuf.p), r, U32,
                                                                 ldu);
  } else {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(apply_basis_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      apply_basis_kernel<double2><<<grid, kAR, smem, h->stream>>>(Dp, ldd, m, n, static_cast<double2*>(wbuf.p), r,
                                                                  U64, ldu);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: basis");
  ++h->launches;
  e = cudaStreamSynchronize(h->stream);  // wbuf is freed on scope exit
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: basis");
  return MROM_OK;
}

// Galerkin projection onto the basis U (n x Rt row-major; r_dirs = per-direction column
// blocks, or all zero for one shared basis) and creation of the reduced object.
mrom_status project_basis(mrom_ctx* h, const mrom_fom* fom, const double2* U, int r, const int32_t* r_dirs,
                          mrom_rom_t* out, const double2* Kin_r = nullptr, const float2* U32in = nullptr) {
  const int64_t n = fom->n;
  cudaStream_t st = h->stream;
  auto launch_grid = [](int64_t work) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(65535 * 4, (work + 255) / 256)); };
  const int ng = 2 * r + 3;
  DevBuf Y, Oc, small, phi, em;
  // K U in float64 feeds the float64 products and the certificate's residual basis
  const bool need_y64 = h->projection_precision != MROM_MIXED || fom_has_certificate(fom);
  cudaError_t e = need_y64 ? cudaMalloc(&Y.p, (size_t)n * r * sizeof(double2)) : cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&Oc.p, (size_t)n * 3 * sizeof(double2));
  const size_t nsmall = 3 * (size_t)r * r + 3 * (size_t)r + 9 + (size_t)ng * ng;
  if (e == cudaSuccess) e = cudaMalloc(&small.p, nsmall * sizeof(double2));
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: allocation");
  double2* Kr = static_cast<double2*>(small.p);
  double2* Cr = Kr + (size_t)r * r;
  double2* Me = Cr + (size_t)r * r;
  double2* Bm = Me + (size_t)r * r;
  double2* c00c = Bm + 3 * (size_t)r;
  double2* Gm = c00c + 9;
  if (need_y64) {
    spmm_csr_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(fom->K_rowptr, fom->K_col, fom->K_val, n, U, r,
                                                                      nullptr, static_cast<double2*>(Y.p));
    ++h->launches;
  }
  complexify_o_kernel<<<launch_grid(3 * n), 256, 0, st>>>(fom->o, n, static_cast<double2*>(Oc.p));
  ++h->launches;
  e = cudaGetLastError();
  const double2* Yp = static_cast<const double2*>(Y.p);
  const double2* Op = static_cast<const double2*>(Oc.p);
  const bool has_me = fom->M_diag && fom->eps != 0.0;
  if (h->projection_precision == MROM_MIXED) {
    // K U, K_r, C_r, eps M_r and b in single precision (complex64 SpMM and Gram products with
    // complex64 accumulation over each CTA's rows, partials summed in float64)
    DevBuf U32, Y32, O32, K32, c32, m32;
    int32_t nnz_host = 0;
    e = cudaMemcpy(&nnz_host, fom->K_rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && !U32in) e = cudaMalloc(&U32.p, (size_t)n * r * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&Y32.p, (size_t)n * r * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&O32.p, (size_t)n * 3 * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&K32.p, (size_t)nnz_host * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c32.p, (size_t)n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m32.p, (size_t)n * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: single-precision buffers");
    if (!U32in)
      to_f32_kernel<<<launch_grid(2 * n * r), 256, 0, st>>>(reinterpret_cast<const double*>(U), 2 * n * r, 1.0,
                                                            static_cast<float*>(U32.p));
    to_f32_kernel<<<launch_grid(6 * n), 256, 0, st>>>(reinterpret_cast<const double*>(Op), 6 * n, 1.0,
                                                      static_cast<float*>(O32.p));
    to_f32_kernel<<<launch_grid(nnz_host), 256, 0, st>>>(fom->K_val, nnz_host, 1.0, static_cast<float*>(K32.p));
    to_f32_kernel<<<launch_grid(n), 256, 0, st>>>(fom->C_diag, n, 1.0, static_cast<float*>(c32.p));
    if (has_me)
      to_f32_kernel<<<launch_grid(n), 256, 0, st>>>(fom->M_diag, n, fom->eps, static_cast<float*>(m32.p));
    spmm_csr_f32_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(
        fom->K_rowptr, fom->K_col, static_cast<float*>(K32.p), n, U32in ? U32in : static_cast<float2*>(U32.p), r,
        static_cast<float2*>(Y32.p));
    h->launches += (has_me ? 6 : 5) - (U32in ? 1 : 0);
    e = cudaGetLastError();
    const auto* u32 = U32in ? U32in : static_cast<const float2*>(U32.p);
    // the Gram products on the tensor cores (tcgen05, 3 x TF32 split, FP32 accumulation per CTA)
    if (e == cudaSuccess) e = tall_gram_tc(h, u32, r, static_cast<float2*>(Y32.p), r, nullptr, n, Kr, r);
    if (e == cudaSuccess) {
      symmetrize_kernel<<<(r * r + 255) / 256, 256, 0, st>>>(Kr, r);
      ++h->launches;
    }
    if (e == cudaSuccess) e = tall_gram_tc(h, u32, r, u32, r, static_cast<float*>(c32.p), n, Cr, r);
    if (e == cudaSuccess && has_me) e = tall_gram_tc(h, u32, r, u32, r, static_cast<float*>(m32.p), n, Me, r);
    if (e == cudaSuccess)
      e = tall_gram_tc(h, u32, r, static_cast<float2*>(O32.p), 3, static_cast<float*>(c32.p), n, Bm, 3);
  } else {
    // K_r = U^H (K U) is Hermitian (K is symmetric): upper tiles, mirrored, then symmetrised
    if (e == cudaSuccess) e = tall_gram(h, U, r, 1, r, Yp, r, 1, r, nullptr, 0, n, true, Kr, r);
    if (e == cudaSuccess) {
      symmetrize_kernel<<<(r * r + 255) / 256, 256, 0, st>>>(Kr, r);
      ++h->launches;
    }
    // C_r, B = U^H C O and c00 = O^T C O from one Hermitian Gram of [U | O] with weight C
    {
      DevBuf UO, Guo;
      const int m = r + 3;
      if (e == cudaSuccess) e = cudaMalloc(&UO.p, (size_t)n * m * sizeof(double2));
      if (e == cudaSuccess) e = cudaMalloc(&Guo.p, (size_t)m * m * sizeof(double2));
      if (e == cudaSuccess) {
        concat_uo_kernel<<<launch_grid((int64_t)m * n), 256, 0, st>>>(U, r, Op, n, static_cast<double2*>(UO.p));
        ++h->launches;
        e = cudaGetLastError();
      }
      const auto* uo = static_cast<const double2*>(UO.p);
      if (e == cudaSuccess)
        e = tall_gram(h, uo, m, 1, m, uo, m, 1, m, fom->C_diag, 1, n, true, static_cast<double2*>(Guo.p), m);
      if (e == cudaSuccess) {
        split_uo_kernel<<<(m * m + 255) / 256, 256, 0, st>>>(static_cast<double2*>(Guo.p), r, Cr, Bm, c00c);
        ++h->launches;
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // UO and Guo are freed on scope exit
    }
    if (e == cudaSuccess && has_me) {
      e = cudaMalloc(&em.p, n * sizeof(double));
      if (e == cudaSuccess) {
        scale_kernel<<<launch_grid(n), 256, 0, st>>>(fom->M_diag, fom->eps, n, static_cast<double*>(em.p));
        ++h->launches;
        e = cudaGetLastError();
      }
      // Me = U^H diag(eps m) U  (added to the reduced system only, Eq. (17))
      if (e == cudaSuccess) e = tall_gram(h, U, r, 1, r, U, r, 1, r, static_cast<double*>(em.p), 1, n, true, Me, r);
    }
  }
  if (e == cudaSuccess && h->projection_precision == MROM_MIXED)
    e = tall_gram(h, Op, 3, 1, 3, Op, 3, 1, 3, fom->C_diag, 1, n, true, c00c, 3);
  const bool cert = fom_has_certificate(fom);
  if (e == cudaSuccess && cert) {
    e = cudaMalloc(&phi.p, (size_t)n * ng * sizeof(double2));
    if (e == cudaSuccess) {
      build_phi_kernel<<<launch_grid((int64_t)ng * n), 256, 0, st>>>(fom->o, fom->C_diag, fom->M_diag, fom->eps, Yp, U,
                                                                     r, n, static_cast<double2*>(phi.p));
      ++h->launches;
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && cert && fom->X_rowptr) {
    // sparse X: G = Phi^H (X^-1 Phi), the representers by PCG, then the Hermitian average
    DevBuf xphi;
    e = cudaMalloc(&xphi.p, (size_t)n * ng * sizeof(double2));
    if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: allocation");
    const mrom_status rs = riesz_solve(h, fom, static_cast<double2*>(phi.p), ng, static_cast<double2*>(xphi.p), nullptr);
    if (rs != MROM_OK) return rs;
    e = tall_gram(h, static_cast<double2*>(phi.p), ng, 1, ng, static_cast<double2*>(xphi.p), ng, 1, ng, nullptr, 0, n,
                  false, Gm, ng);
    if (e == cudaSuccess) {
      symmetrize_kernel<<<(ng * ng + 255) / 256, 256, 0, st>>>(Gm, ng);
      ++h->launches;
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // xphi is freed on scope exit
  } else if (e == cudaSuccess && cert) {
    // X^-1 once (the Gram kernel would otherwise divide for every staged element)
    DevBuf xinv;
    if (e == cudaSuccess) e = cudaMalloc(&xinv.p, (size_t)n * sizeof(double));
    if (e == cudaSuccess) {
      recip_kernel<<<launch_grid(n), 256, 0, st>>>(fom->X_diag, n, static_cast<double*>(xinv.p));
      ++h->launches;
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = tall_gram(h, static_cast<double2*>(phi.p), ng, 1, ng, static_cast<double2*>(phi.p), ng, 1, ng,
                    static_cast<double*>(xinv.p), 1, n, true, Gm, ng);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: projection");
  std::vector<double2> c00h(9);
  e = cudaMemcpy(c00h.data(), c00c, 9 * sizeof(double2), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: read-back");
  double c00[9];
  for (int k = 0; k < 9; ++k) c00[k] = c00h[k].x;
  mrom_reduced_desc d{};
  d.r = r;
  d.K = Kr;
  d.C = Cr;
  d.Me = has_me ? Me : nullptr;
  d.B = Bm;
  d.K_in = Kin_r;
  d.c00 = c00;
  d.G = cert ? Gm : nullptr;
  d.N0 = fom->N0;
  d.alpha = fom->alpha;
  d.alpha_lb = cert ? fom->alpha_lb : 0.0;
  d.vol_B = fom->vol_B;
  for (int i = 0; i < 3; ++i) d.r_dirs[i] = r_dirs ? r_dirs[i] : 0;
  return mrom_rom_from_reduced(h, &d, out);
}

mrom_status check_fom(mrom_ctx* h, const mrom_fom* fom) {
  if (!fom) return fail(h, MROM_EINVAL, "mrom_project: null argument");
  if (fom->n < 1 || !fom->K_rowptr || !fom->K_col || !fom->K_val || !fom->C_diag || !fom->o)
    return fail(h, MROM_EINVAL, "mrom_project: n, K, C_diag and o are required");
  if (!(fom->alpha > 0) || !std::isfinite(fom->alpha) || !std::isfinite(fom->eps))
    return fail(h, MROM_EINVAL, "mrom_project: alpha must be finite and > 0, eps finite");
  if (fom_has_certificate(fom) && !(fom->alpha_lb > 0))
    return fail(h, MROM_EINVAL, "mrom_project: a certificate needs alpha_lb > 0");
  if (fom->X_rowptr && (!fom->X_col || !fom->X_val))
    return fail(h, MROM_EINVAL, "mrom_project: a sparse X needs X_rowptr, X_col and X_val");
  if (!std::isfinite(fom->X_tol) || fom->X_tol < 0.0 || fom->X_max_iter < 0)
    return fail(h, MROM_EINVAL, "mrom_project: X_tol must be finite and >= 0, X_max_iter >= 0");
  return MROM_OK;
}

}  // namespace
}  // namespace mrom

extern "C" mrom_status mrom_project(mrom_handle h, const mrom_fom* fom, const void* D, int64_t ldd, int32_t n_cols,
                                    double tol_sigma, int32_t r_max, const void* basis_in, int32_t r_in,
                                    mrom_rom_t* out, double* sigma_out, int32_t* r_out) {
  if (!h) return MROM_EINVAL;
  if (!out) return fail(h, MROM_EINVAL, "mrom_project: null argument");
  *out = nullptr;
  mrom_status st = check_fom(h, fom);
  if (st != MROM_OK) return st;
  const int64_t n = fom->n;
  if (!basis_in) {
    if (!D || n_cols < 1 || n_cols > MROM_MAX_SNAPSHOTS || ldd < n)
      return fail(h, MROM_EINVAL, "mrom_project: D needs 1..MROM_MAX_SNAPSHOTS columns and ldd >= n");
    if (!(tol_sigma >= 0.0) || !std::isfinite(tol_sigma))
      return fail(h, MROM_EINVAL, "mrom_project: tol_sigma must be finite and >= 0");
  } else if (r_in < 1 || r_in > MROM_MAX_R) {
    return fail(h, MROM_EINVAL, "mrom_project: r_in must be in [1, MROM_MAX_R]");
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: cudaSetDevice");
  if (basis_in) {
    if (r_out) *r_out = r_in;
    return project_basis(h, fom, static_cast<const double2*>(basis_in), r_in, nullptr, out);
  }
  const auto* Dp = static_cast<const double2*>(D);
  int r = 0;
  std::vector<double> s;
  std::vector<double2> wh;
  st = gram_eig(h, Dp, ldd, n, n_cols, tol_sigma, std::min<int>(r_max > 0 ? r_max : MROM_MAX_R, MROM_MAX_R), &r, s, wh);
  if (st != MROM_OK) return st;
  if (sigma_out) std::copy(s.begin(), s.end(), sigma_out);
  if (r_out) *r_out = r;
  const bool b32 = h->projection_precision == MROM_MIXED && !fom_has_certificate(fom);
  DevBuf Ubuf;
  e = cudaMalloc(&Ubuf.p, (size_t)n * r * (b32 ? sizeof(float2) : sizeof(double2)));
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project: basis allocation");
  if (b32) {
    st = apply_basis(h, Dp, ldd, n, n_cols, wh, r, nullptr, r, static_cast<float2*>(Ubuf.p));
    if (st != MROM_OK) return st;
    return project_basis(h, fom, nullptr, r, nullptr, out, nullptr, static_cast<const float2*>(Ubuf.p));
  }
  st = apply_basis(h, Dp, ldd, n, n_cols, wh, r, static_cast<double2*>(Ubuf.p), r);
  if (st != MROM_OK) return st;
  return project_basis(h, fom, static_cast<const double2*>(Ubuf.p), r, nullptr, out);
}

extern "C" mrom_status mrom_project_dirs(mrom_handle h, const mrom_fom* fom, const void* D, int64_t ldd, int32_t n_s,
                                         double tol_sigma, int32_t r_max, const void* basis_in,
                                         const int32_t* r_dirs_in, mrom_rom_t* out, double* sigma_out,
                                         int32_t* r_dirs_out) {
  if (!h) return MROM_EINVAL;
  if (!out) return fail(h, MROM_EINVAL, "mrom_project_dirs: null argument");
  *out = nullptr;
  mrom_status st = check_fom(h, fom);
  if (st != MROM_OK) return st;
  const int64_t n = fom->n;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project_dirs: cudaSetDevice");
  int32_t rd[3] = {0, 0, 0};
  if (basis_in) {
    if (!r_dirs_in) return fail(h, MROM_EINVAL, "mrom_project_dirs: a basis needs r_dirs_in");
    int rt = 0;
    for (int i = 0; i < 3; ++i) {
      if (r_dirs_in[i] < 1) return fail(h, MROM_EINVAL, "mrom_project_dirs: every direction needs r >= 1");
      rd[i] = r_dirs_in[i];
      rt += rd[i];
    }
    if (rt > MROM_MAX_R) return fail(h, MROM_EINVAL, "mrom_project_dirs: r_1 + r_2 + r_3 exceeds MROM_MAX_R");
    if (r_dirs_out) std::copy(rd, rd + 3, r_dirs_out);
    return project_basis(h, fom, static_cast<const double2*>(basis_in), rt, rd, out);
  }
  if (!D || n_s < 1 || 3 * n_s > MROM_MAX_SNAPSHOTS || ldd < n)
    return fail(h, MROM_EINVAL, "mrom_project_dirs: D needs 3 x n_s columns (3 n_s <= MROM_MAX_SNAPSHOTS), ldd >= n");
  if (!(tol_sigma >= 0.0) || !std::isfinite(tol_sigma))
    return fail(h, MROM_EINVAL, "mrom_project_dirs: tol_sigma must be finite and >= 0");
  const auto* Dp = static_cast<const double2*>(D);
  std::vector<double2> wh[3];
  {
    std::vector<double> sv[3];
    const int cap = std::min<int>(r_max > 0 ? r_max : MROM_MAX_R, MROM_MAX_R);
    st = gram_eig_many(h, 3, Dp, ldd, n, n_s, tol_sigma, cap, rd, sv, wh);  // the three directions
    if (st != MROM_OK) return st;
    if (sigma_out)
      for (int i = 0; i < 3; ++i) std::copy(sv[i].begin(), sv[i].end(), sigma_out + (size_t)i * n_s);
  }
  const int rt = rd[0] + rd[1] + rd[2];
  if (rt > MROM_MAX_R) return fail(h, MROM_EINVAL, "mrom_project_dirs: r_1 + r_2 + r_3 exceeds MROM_MAX_R");
  if (r_dirs_out) std::copy(rd, rd + 3, r_dirs_out);
  // the mixed mode without a certificate needs the basis only in complex64
  const bool b32 = h->projection_precision == MROM_MIXED && !fom_has_certificate(fom);
  DevBuf Ubuf;
  e = cudaMalloc(&Ubuf.p, (size_t)n * rt * (b32 ? sizeof(float2) : sizeof(double2)));
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project_dirs: basis allocation");
  int off = 0;
  for (int i = 0; i < 3; ++i) {
    st = b32 ? apply_basis(h, Dp + (size_t)i * n_s * ldd, ldd, n, n_s, wh[i], rd[i], nullptr, rt,
                           static_cast<float2*>(Ubuf.p) + off)
             : apply_basis(h, Dp + (size_t)i * n_s * ldd, ldd, n, n_s, wh[i], rd[i],
                           static_cast<double2*>(Ubuf.p) + off, rt);
    if (st != MROM_OK) return st;
    off += rd[i];
  }
  if (b32) return project_basis(h, fom, nullptr, rt, rd, out, nullptr, static_cast<const float2*>(Ubuf.p));
  return project_basis(h, fom, static_cast<const double2*>(Ubuf.p), rt, rd, out);
}

extern "C" mrom_status mrom_rom_get(mrom_rom_t rom, void* K, void* C, void* Me, void* B, double* c00, void* G) {
  if (!rom) return MROM_EINVAL;
  mrom_ctx* h = rom->ctx;
  const size_t rr = (size_t)rom->r * rom->r;
  const size_t ng = (size_t)(2 * rom->r + 3);
  cudaSetDevice(h->device);
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (dst && e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyDefault);
  };
  cp(K, rom->K, rr * 16);
  cp(C, rom->C, rr * 16);
  if (Me) {
    if (rom->Me) {
      cp(Me, rom->Me, rr * 16);
    } else {
      const std::vector<double2> zeros(rr, make_double2(0.0, 0.0));
      cp(Me, zeros.data(), rr * 16);
    }
  }
  cp(B, rom->B, 3 * (size_t)rom->r * 16);
  if (c00) std::copy(rom->c00, rom->c00 + 9, c00);
  if (G) {
    if (!rom->G) return fail(h, MROM_EINVAL, "mrom_rom_get: object has no Gram matrix");
    cp(G, rom->G, ng * ng * 16);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_rom_get");
  return MROM_OK;
}

extern "C" mrom_status mrom_project_mu(mrom_handle h, const mrom_fom* fom, const mrom_fom_mu* mu, const void* D,
                                       int64_t ldd, int32_t n_cols, double tol_sigma, int32_t r_max,
                                       mrom_rom_t* out, int32_t* r_out, int32_t* m_out) {
  if (!h) return MROM_EINVAL;
  if (!out || !mu) return fail(h, MROM_EINVAL, "mrom_project_mu: null argument");
  *out = nullptr;
  mrom_status st = check_fom(h, fom);
  if (st != MROM_OK) return st;
  const int64_t n = fom->n;
  if (!D || n_cols < 1 || n_cols > MROM_MAX_SNAPSHOTS || ldd < n)
    return fail(h, MROM_EINVAL, "mrom_project_mu: D needs 1..MROM_MAX_SNAPSHOTS columns and ldd >= n");
  if (!(tol_sigma >= 0.0) || !std::isfinite(tol_sigma) || !(mu->tol_static >= 0.0) || !std::isfinite(mu->tol_static))
    return fail(h, MROM_EINVAL, "mrom_project_mu: tolerances must be finite and >= 0");
  if (!mu->Kin_rowptr || !mu->Kin_col || !mu->Kin_val || !mu->x || !mu->kx || !mu->kx_in || !mu->M_static || !mu->O)
    return fail(h, MROM_EINVAL, "mrom_project_mu: K_in, x, kx, kx_in, M_static and O are required");
  if (mu->n_o < 1 || mu->n_o > MROM_MAX_SNAPSHOTS || mu->ldo < n || !std::isfinite(mu->vol_B_mu))
    return fail(h, MROM_EINVAL, "mrom_project_mu: O needs 1..MROM_MAX_SNAPSHOTS columns, ldo >= n, finite vol_B_mu");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project_mu: cudaSetDevice");
  cudaStream_t str = h->stream;
  auto grid_of = [](int64_t work) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(65535 * 4, (work + 255) / 256)); };
  // dynamic basis U (n x r) from the snapshots at the sampled (omega, s)
  const auto* Dp = static_cast<const double2*>(D);
  int r = 0;
  std::vector<double> sv;
  std::vector<double2> wh;
  st = gram_eig(h, Dp, ldd, n, n_cols, tol_sigma, std::min<int>(r_max > 0 ? r_max : MROM_MAX_R, MROM_MAX_R), &r, sv, wh);
  if (st != MROM_OK) return st;
  DevBuf Ubuf, Oc, Vbuf, Y, small;
  e = cudaMalloc(&Ubuf.p, (size_t)n * r * sizeof(double2));
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project_mu: allocation");
  st = apply_basis(h, Dp, ldd, n, n_cols, wh, r, static_cast<double2*>(Ubuf.p), r);
  if (st != MROM_OK) return st;
  const auto* U = static_cast<const double2*>(Ubuf.p);
  // static basis V (n x m) from the static snapshots (real columns)
  const int n_o = mu->n_o;
  e = cudaMalloc(&Oc.p, (size_t)n * n_o * sizeof(double2));
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project_mu: allocation");
  real_cols_kernel<<<grid_of(n * n_o), 256, 0, str>>>(mu->O, mu->ldo, n, n_o, static_cast<double2*>(Oc.p));
  ++h->launches;
  int m = 0;
  st = gram_eig(h, static_cast<double2*>(Oc.p), n, n, n_o, mu->tol_static, MROM_MAX_STATIC, &m, sv, wh);
  if (st != MROM_OK) return st;
  e = cudaMalloc(&Vbuf.p, (size_t)n * m * sizeof(double2));
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project_mu: allocation");
  st = apply_basis(h, static_cast<double2*>(Oc.p), n, n, n_o, wh, m, static_cast<double2*>(Vbuf.p), m);
  if (st != MROM_OK) return st;
  const auto* V = static_cast<const double2*>(Vbuf.p);
  // K_in^r = U^H (K_in U)
  const int wmax = std::max(r, m);
  e = cudaMalloc(&Y.p, (size_t)n * wmax * sizeof(double2));
  const size_t n_small = (size_t)r * r + (size_t)m * m + 3 * (size_t)m + 9;  // K_in^r, then V^H K V, V^H K x, x^T C x
  if (e == cudaSuccess) e = cudaMalloc(&small.p, n_small * sizeof(double2));
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project_mu: allocation");
  auto* Yp = static_cast<double2*>(Y.p);
  auto* Kin_r = static_cast<double2*>(small.p);
  spmm_csr_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, str>>>(mu->Kin_rowptr, mu->Kin_col, mu->Kin_val, n, U, r,
                                                                     nullptr, Yp);
  ++h->launches;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = tall_gram(h, U, r, 1, r, Yp, r, 1, r, nullptr, 0, n, true, Kin_r, r);
  if (e == cudaSuccess) {
    symmetrize_kernel<<<(r * r + 255) / 256, 256, 0, str>>>(Kin_r, r);
    ++h->launches;
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_project_mu: K_in projection");
  st = project_basis(h, fom, U, r, nullptr, out, Kin_r);
  if (st != MROM_OK) return st;
  mrom_rom* rom = *out;
  auto bail = [&](cudaError_t err, const char* what) {
    mrom_rom_free(rom);
    *out = nullptr;
    return cuda_fail(h, err, what);
  };
  // reduced static data, one device block owned by the object:
  // Sout, Sin, Mv, cvv (m x m), kout, kin, cvx (m x 3), Bx (r x 3), BV (r x m)
  const size_t mm = (size_t)m * m, m3 = 3 * (size_t)m;
  const bool cert = fom_has_certificate(fom);
  const int n_ext = 3 + m + 3 * r;
  const size_t n_mu = 4 * mm + 3 * m3 + 3 * (size_t)r + (size_t)r * m + (cert ? (size_t)n_ext * n_ext : 0);
  void* blk = nullptr;
  e = cudaMalloc(&blk, n_mu * sizeof(double2));
  if (e != cudaSuccess) return bail(e, "mrom_project_mu: allocation");
  rom->mu_block = blk;
  MuDev md{};
  auto* q = static_cast<double2*>(blk);
  double2* Sout = q; q += mm;
  double2* Sin = q; q += mm;
  double2* Mv = q; q += mm;
  double2* cvv = q; q += mm;
  double2* kout = q; q += m3;
  double2* kin = q; q += m3;
  double2* cvx = q; q += m3;
  double2* Bx = q; q += 3 * (size_t)r;
  double2* BV = q; q += (size_t)r * m;
  double2* Gext = cert ? q : nullptr;
  // scratch in the small block after K_in^r
  double2* Sv = Kin_r + (size_t)r * r;        // m x m
  double2* kv = Sv + mm;                     // m x 3
  double2* cxx = kv + m3;                    // 3 x 3
  DevBuf Xb, KXb, KXinb;
  e = cudaMalloc(&Xb.p, (size_t)n * 3 * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&KXb.p, (size_t)n * 3 * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&KXinb.p, (size_t)n * 3 * sizeof(double2));
  if (e != cudaSuccess) return bail(e, "mrom_project_mu: allocation");
  auto* X3 = static_cast<double2*>(Xb.p);
  auto* KX3 = static_cast<double2*>(KXb.p);
  auto* KXin3 = static_cast<double2*>(KXinb.p);
  complexify_o_kernel<<<grid_of(3 * n), 256, 0, str>>>(mu->x, n, X3);
  complexify_o_kernel<<<grid_of(3 * n), 256, 0, str>>>(mu->kx, n, KX3);
  complexify_o_kernel<<<grid_of(3 * n), 256, 0, str>>>(mu->kx_in, n, KXin3);
  h->launches += 3;
  e = cudaGetLastError();
  // V^H K V and V^H K_in V (Hermitian), Sout = the difference
  if (e == cudaSuccess) {
    spmm_csr_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, str>>>(fom->K_rowptr, fom->K_col, fom->K_val, n, V, m,
                                                                       nullptr, Yp);
    ++h->launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = tall_gram(h, V, m, 1, m, Yp, m, 1, m, nullptr, 0, n, true, Sv, m);
  if (e == cudaSuccess) {
    spmm_csr_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, str>>>(mu->Kin_rowptr, mu->Kin_col, mu->Kin_val, n, V,
                                                                       m, nullptr, Yp);
    ++h->launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = tall_gram(h, V, m, 1, m, Yp, m, 1, m, nullptr, 0, n, true, Sin, m);
  if (e == cudaSuccess) {
    symmetrize_kernel<<<(int)((mm + 255) / 256), 256, 0, str>>>(Sv, m);
    symmetrize_kernel<<<(int)((mm + 255) / 256), 256, 0, str>>>(Sin, m);
    csub_kernel<<<(int)((mm + 255) / 256), 256, 0, str>>>(Sv, Sin, (int)mm, Sout);
    h->launches += 3;
    e = cudaGetLastError();
  }
  // V^H M_s V, V^H C V (Hermitian); V^H (K x), V^H (K_in x), V^H C x; U^H C x, U^H C V; x^T C x
  if (e == cudaSuccess) e = tall_gram(h, V, m, 1, m, V, m, 1, m, mu->M_static, 1, n, true, Mv, m);
  if (e == cudaSuccess) e = tall_gram(h, V, m, 1, m, V, m, 1, m, fom->C_diag, 1, n, true, cvv, m);
  if (e == cudaSuccess) e = tall_gram(h, V, m, 1, m, KX3, 3, 1, 3, nullptr, 0, n, false, kv, 3);
  if (e == cudaSuccess) e = tall_gram(h, V, m, 1, m, KXin3, 3, 1, 3, nullptr, 0, n, false, kin, 3);
  if (e == cudaSuccess) {
    csub_kernel<<<(int)((m3 + 255) / 256), 256, 0, str>>>(kv, kin, (int)m3, kout);
    ++h->launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = tall_gram(h, V, m, 1, m, X3, 3, 1, 3, fom->C_diag, 1, n, false, cvx, 3);
  if (e == cudaSuccess) e = tall_gram(h, U, r, 1, r, X3, 3, 1, 3, fom->C_diag, 1, n, false, Bx, 3);
  if (e == cudaSuccess) e = tall_gram(h, U, r, 1, r, V, m, 1, m, fom->C_diag, 1, n, false, BV, m);
  if (e == cudaSuccess) e = tall_gram(h, X3, 3, 1, 3, X3, 3, 1, 3, fom->C_diag, 1, n, true, cxx, 3);
  // certificate at a permeability scale: G_ext = Phi_ext^H X^-1 Phi_ext
  if (e == cudaSuccess && cert) {
    DevBuf KinUb, Phib, xinv;
    e = cudaMalloc(&KinUb.p, (size_t)n * r * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&Phib.p, (size_t)n * n_ext * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&xinv.p, (size_t)n * sizeof(double));
    if (e == cudaSuccess) {
      spmm_csr_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, str>>>(fom->K_rowptr, fom->K_col, fom->K_val, n, U,
                                                                         r, nullptr, Yp);
      spmm_csr_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, str>>>(mu->Kin_rowptr, mu->Kin_col, mu->Kin_val, n,
                                                                         U, r, nullptr,
                                                                         static_cast<double2*>(KinUb.p));
      build_phi_ext_kernel<<<grid_of((int64_t)n * n_ext), 256, 0, str>>>(
          X3, V, m, U, Yp, static_cast<double2*>(KinUb.p), r, fom->C_diag, fom->M_diag, fom->eps, n,
          static_cast<double2*>(Phib.p));
      if (!fom->X_rowptr) {
        recip_kernel<<<grid_of(n), 256, 0, str>>>(fom->X_diag, n, static_cast<double*>(xinv.p));
        ++h->launches;
      }
      h->launches += 3;
      e = cudaGetLastError();
    }
    const auto* Phi = static_cast<const double2*>(Phib.p);
    if (e == cudaSuccess && fom->X_rowptr) {
      // sparse X: the representers X^-1 Phi_ext by PCG, G_ext = Phi_ext^H (X^-1 Phi_ext), Hermitian average
      DevBuf xphi;
      e = cudaMalloc(&xphi.p, (size_t)n * n_ext * sizeof(double2));
      if (e == cudaSuccess) {
        const mrom_status rs = riesz_solve(h, fom, Phi, n_ext, static_cast<double2*>(xphi.p), nullptr);
        if (rs != MROM_OK) {
          mrom_rom_free(rom);
          *out = nullptr;
          return rs;
        }
        e = tall_gram(h, Phi, n_ext, 1, n_ext, static_cast<double2*>(xphi.p), n_ext, 1, n_ext, nullptr, 0, n, false,
                      Gext, n_ext);
      }
      if (e == cudaSuccess) {
        symmetrize_kernel<<<(n_ext * n_ext + 255) / 256, 256, 0, str>>>(Gext, n_ext);
        ++h->launches;
        e = cudaGetLastError();
      }
    } else if (e == cudaSuccess) {
      e = tall_gram(h, Phi, n_ext, 1, n_ext, Phi, n_ext, 1, n_ext, static_cast<double*>(xinv.p), 1, n, true, Gext,
                    n_ext);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(str);
  }
  std::vector<double2> cxx_h(9);
  if (e == cudaSuccess) e = cudaMemcpy(cxx_h.data(), cxx, 9 * sizeof(double2), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bail(e, "mrom_project_mu: static projection");
  const double a3 = fom->alpha * fom->alpha * fom->alpha;
  md.Sout = Sout;
  md.Sin = Sin;
  md.Mv = Mv;
  md.kout = kout;
  md.kin = kin;
  md.cvx = cvx;
  md.cvv = cvv;
  md.Bx = Bx;
  md.BV = BV;
  for (int k = 0; k < 9; ++k) md.cxx[k] = cxx_h[k].x;
  md.nB = a3 * fom->vol_B;
  md.mB = a3 * mu->vol_B_mu;
  md.alpha3 = a3;
  md.m = m;
  md.r = r;
  md.Gext = Gext;
  md.next = cert ? n_ext : 0;
  rom->mu = md;
  // the object's B, c00 and N0 become those of the reduced static problem at s = 1
  DevBuf inst;
  e = cudaMalloc(&inst.p, sizeof(MuDev) + sizeof(RomDev) + (3 * (size_t)r + 3 * (size_t)m) * sizeof(double2) + 64);
  if (e != cudaSuccess) return bail(e, "mrom_project_mu: allocation");
  auto* dmu = static_cast<MuDev*>(inst.p);
  auto* drec = reinterpret_cast<RomDev*>(dmu + 1);
  auto* dscr = reinterpret_cast<double2*>(drec + 1);
  MuDev md1 = md;
  md1.Bdst = rom->B;
  md1.dBdst = dscr;
  md1.ydst = dscr + 3 * (size_t)r;
  if (cert && rom->GKK) {  // the object's certificate blocks become those of G_ext at s = 1
    md1.GKKdst = rom->GKK;
    md1.GSkdst = rom->GSk;
    md1.gsKdst = rom->gsK;
    md1.gsCdst = rom->gsC;
  } else {
    md1.Gext = nullptr;
  }
  e = cudaMemcpyAsync(dmu, &md1, sizeof(MuDev), cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess) e = launch_mu_instance(dmu, 1, m, nullptr, false, drec, nullptr, h->d_status, str);
  if (e == cudaSuccess && md1.Gext) {
    e = launch_mu_cert(dmu, 1, nullptr, drec, str);
    ++h->launches;
  }
  RomDev rec{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&rec, drec, sizeof(RomDev), cudaMemcpyDeviceToHost, str);
  if (e == cudaSuccess) e = cudaStreamSynchronize(str);
  if (e != cudaSuccess) return bail(e, "mrom_project_mu: static state at s = 1");
  ++h->launches;
  st = mrom_synchronize(h);
  if (st != MROM_OK) {
    mrom_rom_free(rom);
    *out = nullptr;
    return st;
  }
  std::copy(rec.c00, rec.c00 + 9, rom->c00);
  std::copy(rec.N0, rec.N0 + 9, rom->N0);
  if (md1.Gext) std::copy(rec.gss, rec.gss + 9, rom->gss);
  if (r_out) *r_out = r;
  if (m_out) *m_out = m;
  return MROM_OK;
}
