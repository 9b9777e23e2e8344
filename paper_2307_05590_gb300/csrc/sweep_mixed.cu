// Mixed-precision batched sweep: complex64 elimination + float64 iterative refinement.
//
// Same outputs as sweep_fp64.cu (R of Eq. (18), I of Eq. (19), Delta of Lemma 4.2).
// On GB300 the FP32 pipe is about 60x faster than the FP64 pipe, so the O(r^3)
// elimination of the reduced system (Eq. (17)) runs in complex64; the solution is
// then refined n_refine times in float64:
//   res = i w B - (K + Me - i w C) X      (float64, K, C, Me read from L2)
//   solve L U d = res in complex64 with the same factors,  X <- X + d,
// and the quadratic forms and the certificate (where I and Delta cancel at high
// omega) are evaluated in float64 exactly as in the float64 sweep.  Without
// pivoting the complex64 elimination is as stable as the float64 one (A is
// sectorial); each refinement step multiplies the error by about kappa(A) * 6e-8.
#include "mrom_internal.h"

#include <algorithm>
#include <numeric>

namespace mrom {
namespace {

constexpr int kT = 256;
constexpr int kW = kT / 32;
constexpr int kRed = 45;
constexpr int kSplit = 4;

__device__ __forceinline__ float2 f_msub(float2 c, float2 a, float2 b) {
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 f_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 f_recip(float2 a, int* status) {
  const float d = fmaf(a.x, a.x, a.y * a.y);
  if (!(d > 0.0f) || !isfinite(d)) {
    atomicOr(status, kStatusSingular);
    return make_float2(__int_as_float(0x7fc00000), 0.0f);
  }
  const float id = 1.0f / d;
  return make_float2(a.x * id, -a.y * id);
}
__device__ __forceinline__ double2 c_conj_mac(double2 c, double2 a, double2 b) {  // c + conj(a) b
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}

__host__ __device__ __forceinline__ size_t region_bytes(int r) {
  const size_t lu = (size_t)8 * r * (r + 3);
  const size_t forms = (size_t)16 * (9 * (size_t)r + (size_t)r * (r + 1) / 2);
  return lu > forms ? lu : forms;
}

__global__ void __launch_bounds__(kT, 2)
sweep_mixed_kernel(const RomDev* __restrict__ objs, const SweepTask* __restrict__ tasks, int n_tasks,
                   int* __restrict__ counter, const double* __restrict__ omega, int omega_stride, int n_refine,
                   double* __restrict__ Rout, double* __restrict__ Iout, double* __restrict__ Dout,
                   int* __restrict__ status, int n_w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    if (tid == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= n_tasks) break;
    const SweepTask task = tasks[t];
    const RomDev& ob = objs[task.obj];
    const int r = ob.r, S = task.nw, ld = r + 3;
    const bool want_cert = (Dout != nullptr) && ob.has_cert;
    const size_t reg = region_bytes(r);
    unsigned char* base = smem_raw;
    double2* Xm = reinterpret_cast<double2*>(base + (size_t)S * reg);   // S * r * 3 float64 solutions
    float2* Inv = reinterpret_cast<float2*>(Xm + (size_t)S * r * 3);    // S * r
    double* Ws = reinterpret_cast<double*>(Inv + (size_t)S * r);        // S
    double* Red = Ws + S;                                               // S * kRed * kSplit
    auto Af = [&](int s) { return reinterpret_cast<float2*>(base + (size_t)s * reg); };
    auto Ad = [&](int s) { return reinterpret_cast<double2*>(base + (size_t)s * reg); };

    for (int s = tid; s < S; s += kT) {
      const double w = omega[(size_t)task.obj * omega_stride + task.w0 + s];
      const bool ok = (w > 0.0) && isfinite(w);
      if (!ok) atomicOr(status, kStatusBadOmega);
      Ws[s] = ok ? w : __longlong_as_double(0x7ff8000000000000LL);
    }
    __syncthreads();

    // ---- 1. [A | i w B] rounded to complex64
    for (int idx = tid; idx < S * r * ld; idx += kT) {
      const int s = idx / (r * ld), e = idx - (idx / (r * ld)) * (r * ld);
      const int i = e / ld, j = e - (e / ld) * ld;
      const double w = Ws[s];
      double2 v;
      if (j < r) {
        double2 k = ob.K[i * r + j];
        if (ob.Me) {
          const double2 m = ob.Me[i * r + j];
          k.x += m.x;
          k.y += m.y;
        }
        const double2 c = ob.C[i * r + j];
        v = make_double2(fma(w, c.y, k.x), fma(-w, c.x, k.y));
      } else {
        const double2 b = ob.B[i * 3 + (j - r)];
        v = make_double2(-w * b.y, w * b.x);
      }
      const float2 f = make_float2((float)v.x, (float)v.y);
      Af(s)[e] = f;
      if (e == 0) Inv[(size_t)s * r] = f_recip(f, status);
    }
    __syncthreads();

    // ---- 2. complex64 elimination without pivoting
    for (int k = 0; k < r - 1; ++k) {
      const int m = r - k - 1;
      for (int idx = tid; idx < S * m; idx += kT) {
        const int s = idx / m, i = k + 1 + (idx - (idx / m) * m);
        float2* a = Af(s);
        a[i * ld + k] = f_mul(a[i * ld + k], Inv[(size_t)s * r + k]);
      }
      __syncthreads();
      const int nc = ld - k - 1, per = m * nc;
      for (int idx = tid; idx < S * per; idx += kT) {
        const int s = idx / per, e = idx - (idx / per) * per;
        const int i = k + 1 + e / nc, j = k + 1 + (e - (e / nc) * nc);
        float2* a = Af(s);
        const float2 v = f_msub(a[i * ld + j], a[i * ld + k], a[k * ld + j]);
        a[i * ld + j] = v;
        if (e == 0) Inv[(size_t)s * r + k + 1] = f_recip(v, status);
      }
      __syncthreads();
    }

    // ---- 3./4. back substitution, then n_refine float64 refinement steps; one warp per
    // (system, right-hand side); the residual goes through the complex64 factors
    for (int sj = warp; sj < S * 3; sj += kW) {
      const int s = sj / 3, j = sj - (sj / 3) * 3;
      float2* a = Af(s);
      const float2* inv = Inv + (size_t)s * r;
      double2* x = Xm + (size_t)s * r * 3;
      const double w = Ws[s];
      for (int k = r - 1; k >= 0; --k) {
        const float2 xk = f_mul(a[k * ld + r + j], inv[k]);
        for (int i = lane; i < k; i += 32) a[i * ld + r + j] = f_msub(a[i * ld + r + j], a[i * ld + k], xk);
        if (lane == 0) x[k * 3 + j] = make_double2(xk.x, xk.y);
        __syncwarp();
      }
      for (int it = 0; it < n_refine; ++it) {
        // res_i = i w b_i - sum_b (K + Me - i w C)_ib x_b, with (K + Me)_ib = conj((K + Me)_bi)
        for (int i = lane; i < r; i += 32) {
          const double2 bi = ob.B[i * 3 + j];
          double2 res = make_double2(-w * bi.y, w * bi.x);
          for (int b = 0; b < r; ++b) {
            double2 k = ob.K[b * r + i];
            if (ob.Me) {
              const double2 mm = ob.Me[b * r + i];
              k.x += mm.x;
              k.y += mm.y;
            }
            const double2 c = ob.C[b * r + i];
            // A_ib = conj(k) - i w conj(c) = (k.x - w c.y) + i (-k.y - w c.x)
            const double2 aib = make_double2(fma(-w, c.y, k.x), fma(-w, c.x, -k.y));
            const double2 xb = x[b * 3 + j];
            res.x = fma(-aib.x, xb.x, fma(aib.y, xb.y, res.x));
            res.y = fma(-aib.x, xb.y, fma(-aib.y, xb.x, res.y));
          }
          a[i * ld + r + j] = make_float2((float)res.x, (float)res.y);
        }
        __syncwarp();
        // L y = res (unit lower, multipliers below the diagonal)
        for (int k = 0; k < r; ++k) {
          const float2 yk = a[k * ld + r + j];
          for (int i = k + 1 + lane; i < r; i += 32) a[i * ld + r + j] = f_msub(a[i * ld + r + j], a[i * ld + k], yk);
          __syncwarp();
        }
        // U d = y, x += d
        for (int k = r - 1; k >= 0; --k) {
          const float2 dk = f_mul(a[k * ld + r + j], inv[k]);
          for (int i = lane; i < k; i += 32) a[i * ld + r + j] = f_msub(a[i * ld + r + j], a[i * ld + k], dk);
          if (lane == 0) {
            double2 xk = x[k * 3 + j];
            xk.x += dk.x;
            xk.y += dk.y;
            x[k * 3 + j] = xk;
          }
          __syncwarp();
        }
      }
    }
    __syncthreads();

    // ---- 5. float64 forms and certificate (as in the float64 sweep); the region of system s
    // now holds Y[mm][a][j] (9 r) and the packed upper triangle of G~ (float64)
    const int nm = want_cert ? 3 : 2;
    const int half = (r + 1) / 2;
    auto tri = [r](int b, int a) { return b * r - (b * (b - 1)) / 2 + (a - b); };
    if (want_cert) {
      const int ntri = r * (r + 1) / 2;
      for (int idx = tid; idx < S * ntri; idx += kT) {
        const int s = idx / ntri;
        int e = idx - s * ntri;
        int b = 0;
        while (e >= r - b) {
          e -= r - b;
          ++b;
        }
        const int a = b + e;
        const double w = Ws[s], w2 = w * w;
        const double2 gk = ob.GKK[b * r + a], gc = ob.GCC[b * r + a], sk = ob.GSk[b * r + a];
        Ad(s)[9 * r + tri(b, a)] = make_double2(fma(w2, gc.x, fma(-w, sk.y, gk.x)), fma(w2, gc.y, fma(w, sk.x, gk.y)));
      }
      __syncthreads();
    }
    for (int idx = tid; idx < S * nm * half * 3; idx += kT) {
      const int s = idx / (nm * half * 3);
      int e = idx - s * nm * half * 3;
      const int mm = e / (half * 3);
      e -= mm * half * 3;
      const int pr = e / 3, j = e - (e / 3) * 3;
      const double2* p = Xm + (size_t)s * r * 3;
      double2* ys = Ad(s);
      const double2* gt = ys + 9 * r;
      const double2* M = mm == 0 ? ob.K : ob.C;
      for (int side = 0; side < 2; ++side) {
        const int a = side == 0 ? pr : r - 1 - pr;
        if (side == 1 && a == pr) break;
        double2 y = make_double2(0.0, 0.0);
        if (mm < 2) {
          for (int b = 0; b < a; ++b) y = c_conj_mac(y, M[b * r + a], p[b * 3 + j]);
          const double2 d = M[a * r + a];
          y = c_conj_mac(y, make_double2(0.5 * d.x, 0.5 * d.y), p[a * 3 + j]);
        } else {
          for (int b = 0; b < a; ++b) y = c_conj_mac(y, gt[tri(b, a)], p[b * 3 + j]);
          const double2 d = gt[tri(a, a)];
          y = c_conj_mac(y, make_double2(0.5 * d.x, 0.5 * d.y), p[a * 3 + j]);
        }
        ys[(mm * r + a) * 3 + j] = y;
      }
    }
    __syncthreads();
    const int nq = want_cert ? kRed : 27;
    for (int idx = tid; idx < S * nq * kSplit; idx += kT) {
      const int s = idx / (nq * kSplit);
      const int e = idx - s * nq * kSplit;
      int q = e / kSplit;
      const int part = e - q * kSplit;
      if (!want_cert && q >= 18) q += 9;
      const int a0 = (r * part) / kSplit, a1 = (r * (part + 1)) / kSplit;
      const double2* p = Xm + (size_t)s * r * 3;
      double acc = 0.0;
      if (q < 27) {
        const int i = (q % 9) / 3, j = q % 3;
        const double2* y = Ad(s) + (q / 9) * r * 3;
        for (int a = a0; a < a1; ++a) {
          const double2 pa = p[a * 3 + i], ya = y[a * 3 + j];
          acc = fma(pa.x, ya.x, fma(pa.y, ya.y, acc));
        }
      } else if (q < 36) {
        const int i = (q - 27) / 3, j = (q - 27) % 3;
        for (int a = a0; a < a1; ++a) {
          const double2 b = ob.B[a * 3 + i], pa = p[a * 3 + j];
          acc = fma(b.x, pa.x, fma(b.y, pa.y, acc));
        }
      } else {
        const int i = (q - 36) / 3, j = (q - 36) % 3;
        const double w = Ws[s], w2 = w * w;
        for (int a = a0; a < a1; ++a) {
          const double2 gk = ob.gsK[i * r + a], gc = ob.gsC[i * r + a], pa = p[a * 3 + j];
          const double cx = fma(-w, gk.y, w2 * gc.x), cy = fma(w, gk.x, w2 * gc.y);
          acc = fma(cx, pa.x, fma(-cy, pa.y, acc));
        }
      }
      Red[((size_t)s * kRed + q) * kSplit + part] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < S * 9; idx += kT) {
      const int s = idx / 9, ij = idx - (idx / 9) * 9;
      const int i = ij / 3, j = ij - (ij / 3) * 3, ji = j * 3 + i;
      const double* rp = Red + (size_t)s * kRed * kSplit;
      auto red = [rp](int q) {
        double v = 0.0;
#pragma unroll
        for (int k = 0; k < kSplit; ++k) v += rp[q * kSplit + k];
        return v;
      };
      const double w = Ws[s];
      const size_t o = ((size_t)task.obj * n_w + task.w0 + s) * 9 + ij;
      if (Rout) Rout[o] = fma(-0.25 * ob.alpha3, red(ij) + red(ji), ob.N0[ij]);
      if (Iout)
        Iout[o] = 0.25 * ob.alpha3 * w * (ob.c00[ij] + red(9 + ij) + red(9 + ji) + red(27 + ij) + red(27 + ji));
      if (Dout) {
        if (want_cert) {
          const double w2 = w * w;
          const double cij = fma(w2, ob.gss[ij], red(18 + ij) + red(18 + ji) + red(36 + ij) + red(36 + ji));
          const double ni = fma(w2, ob.gss[i * 4], 2.0 * (red(18 + i * 4) + red(36 + i * 4)));
          const double nj = fma(w2, ob.gss[j * 4], 2.0 * (red(18 + j * 4) + red(36 + j * 4)));
          Dout[o] = ob.cert_scale * (ni + nj - cij);
        } else {
          Dout[o] = __longlong_as_double(0x7ff8000000000000LL);
        }
      }
    }
  }
}

size_t mixed_bytes_per_system(int r) {
  return region_bytes(r) + 16 * 3 * (size_t)r + 8 * (size_t)r + 8 * (1 + (size_t)kRed * kSplit);
}

}  // namespace
}  // namespace mrom

using namespace mrom;

extern "C" mrom_status mrom_sweep_mixed(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, const double* omega,
                                        int32_t n_w, int32_t omega_stride, int32_t n_refine, double* R, double* I,
                                        double* Delta) {
  if (!h) return MROM_EINVAL;
  if (!roms || n_obj < 1 || n_w < 1 || !omega || n_refine < 0 || n_refine > 8)
    return fail(h, MROM_EINVAL, "mrom_sweep_mixed: bad arguments (n_refine in 0..8)");
  if (omega_stride != 0 && omega_stride < n_w)
    return fail(h, MROM_EINVAL, "mrom_sweep_mixed: omega_stride must be 0 or >= n_w");
  for (int o = 0; o < n_obj; ++o) {
    if (!roms[o] || roms[o]->ctx != h) return fail(h, MROM_EINVAL, "mrom_sweep_mixed: invalid object");
    if (roms[o]->r_dirs[0] + roms[o]->r_dirs[1] + roms[o]->r_dirs[2] > 0)
      return fail(h, MROM_ENOTSUP, "mrom_sweep_mixed: objects with one basis per direction are swept by mrom_sweep");
    if (Delta && !roms[o]->has_cert)
      return fail(h, MROM_EINVAL, "mrom_sweep_mixed: Delta requested but an object has no Gram matrix");
  }
  if (!R && !I && !Delta) return MROM_OK;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep_mixed: cudaSetDevice");
  int per_sm = 0;
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
  const size_t budget = std::min<size_t>(h->smem_optin, (size_t)per_sm / 2) - 2048;
  std::vector<RomDev> objs(n_obj);
  std::vector<SweepTask> tasks;
  std::vector<double> cost;
  size_t smem = 0;
  for (int o = 0; o < n_obj; ++o) {
    objs[o] = rom_record(roms[o]);
    const int r = roms[o]->r;
    const size_t per = mixed_bytes_per_system(r);
    if (per > budget) return fail(h, MROM_ENOTSUP, "mrom_sweep_mixed: r too large for the mixed sweep");
    const int S = std::min<int>(n_w, (int)(budget / per));
    const double rr = r;
    for (int w0 = 0; w0 < n_w; w0 += S) {
      const int nw = std::min(S, n_w - w0);
      tasks.push_back(SweepTask{o, w0, nw, 0});
      cost.push_back((rr * rr * rr / 40.0 + (54.0 + 12.0 * n_refine) * rr * rr) * nw);
      smem = std::max(smem, per * nw);
    }
  }
  std::vector<int> order(tasks.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<SweepTask> sorted(tasks.size());
  for (size_t k = 0; k < order.size(); ++k) sorted[k] = tasks[order[k]];
  e = cudaFuncSetAttribute(sweep_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sweep_mixed_kernel, kT, smem);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep_mixed: configuration");
  const int grid = std::min<int>((int)sorted.size(), h->num_sms * std::max(occ, 1));
  const size_t bytes = n_obj * sizeof(RomDev) + sorted.size() * sizeof(SweepTask) + 16;
  void* blk = nullptr;
  e = cudaMallocAsync(&blk, bytes, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep_mixed: allocation");
  auto* d_objs = static_cast<RomDev*>(blk);
  auto* d_tasks = reinterpret_cast<SweepTask*>(d_objs + n_obj);
  auto* d_counter = reinterpret_cast<int*>(d_tasks + sorted.size());
  e = cudaMemcpyAsync(d_objs, objs.data(), n_obj * sizeof(RomDev), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tasks, sorted.data(), sorted.size() * sizeof(SweepTask), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) {
    sweep_mixed_kernel<<<grid, kT, smem, h->stream>>>(d_objs, d_tasks, (int)sorted.size(), d_counter, omega,
                                                      omega_stride, n_refine, R, I, Delta, h->d_status, n_w);
    e = cudaGetLastError();
  }
  cudaFreeAsync(blk, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep_mixed: launch");
  ++h->launches;
  return MROM_OK;
}
