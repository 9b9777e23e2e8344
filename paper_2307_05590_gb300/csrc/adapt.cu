// Adaptive PODP (Algorithm 1): certificates on the output grid, the per-interval
// maximum Lambda_n and its frequency, and the greedy snapshot loop.
#include "mrom_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <numeric>

namespace mrom {

// Full-order solves of the adaptive loop when no callback is given: Jacobi-scaled residual
// below 1e-12 (R and I then agree with a direct solve to about 1e-13 on the FIT grids)
constexpr double kAdaptSolveTol = 1e-12;
constexpr int kAdaptSolveMaxIter = 100000;
namespace {

__device__ __forceinline__ bool in_sorted(const double* __restrict__ a, int n, double x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo < n && a[lo] == x;
}

// One CTA per snapshot interval [snaps[n], snaps[n+1]) (snaps ascending).  Over the
// output frequencies in the interval that are not themselves snapshots, find the
// largest max_ij Delta_ij (ties: lowest frequency).  lam[n] = -inf and arg[n] = -1
// when the interval holds no candidate.  omega ascending.
__global__ void __launch_bounds__(256)
interval_max_kernel(const double* __restrict__ Delta, const double* __restrict__ omega, int n_out,
                    const double* __restrict__ snaps, int ns, double* __restrict__ lam, int* __restrict__ arg) {
  const int iv = blockIdx.x;
  const double lo = snaps[iv], hi = snaps[iv + 1];
  // first grid index with omega >= lo, and with omega >= hi
  int a = 0, b = n_out;
  {
    int l = 0, h = n_out;
    while (l < h) { const int mid = (l + h) >> 1; if (omega[mid] < lo) l = mid + 1; else h = mid; }
    a = l;
    l = a;
    h = n_out;
    while (l < h) { const int mid = (l + h) >> 1; if (omega[mid] < hi) l = mid + 1; else h = mid; }
    b = l;
  }
  double best = -INFINITY;
  int bi = -1;
  for (int k = a + threadIdx.x; k < b; k += blockDim.x) {
    if (in_sorted(snaps, ns, omega[k])) continue;
    double v = Delta[(size_t)k * 9];
    for (int q = 1; q < 9; ++q) v = fmax(v, Delta[(size_t)k * 9 + q]);
    if (v > best || (v == best && bi >= 0 && k < bi)) {
      best = v;
      bi = k;
    }
  }
  __shared__ double sv[256];
  __shared__ int si[256];
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double v2 = sv[threadIdx.x + s];
      const int i2 = si[threadIdx.x + s];
      const double v1 = sv[threadIdx.x];
      const int i1 = si[threadIdx.x];
      if (i2 >= 0 && (i1 < 0 || v2 > v1 || (v2 == v1 && i2 < i1))) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    lam[iv] = sv[0];
    arg[iv] = si[0];
  }
}


}  // namespace
}  // namespace mrom

using namespace mrom;

extern "C" mrom_status mrom_adapt(mrom_handle h, const mrom_fom* fom, const double* omega0, int32_t ns0,
                                  const void* D0, mrom_snapshot_cb cb, void* user, const double* omega_out,
                                  int32_t n_out, const mrom_adapt_opts* opts, mrom_rom_t* out, double* lambda_hist,
                                  int32_t* k_done, double* omega_snap_out, int32_t* ns_out) {
  if (!h) return MROM_EINVAL;
  if (!fom || !omega0 || ns0 < 2 || (!D0 && cb) || !omega_out || n_out < 2 || !opts || !out)
    return fail(h, MROM_EINVAL, "mrom_adapt: bad arguments");
  if (!fom_has_certificate(fom))
    return fail(h, MROM_EINVAL, "mrom_adapt: the certificate needs fom->X_diag or a sparse X");
  if (opts->n_star < 1 || opts->max_k < 1 || !(opts->tol_delta >= 0.0))
    return fail(h, MROM_EINVAL, "mrom_adapt: n_star >= 1, max_k >= 1 and tol_delta >= 0 are required");
  if (!(opts->theta >= 0.0 && opts->theta <= 1.0))
    return fail(h, MROM_EINVAL, "mrom_adapt: theta must be 0 or in (0, 1]");
  *out = nullptr;
  const int64_t n = fom->n;
  const int ns_cap = ns0 + opts->n_star * std::max(0, opts->max_k - 1);
  if (3 * ns_cap > MROM_MAX_SNAPSHOTS)
    return fail(h, MROM_EINVAL, "mrom_adapt: 3 (ns0 + n_star (max_k - 1)) exceeds MROM_MAX_SNAPSHOTS");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_adapt: cudaSetDevice");
  cudaStream_t st = h->stream;

  std::vector<double> wout(n_out);
  e = cudaMemcpy(wout.data(), omega_out, n_out * sizeof(double), cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_adapt: omega_out read");
  for (int k = 1; k < n_out; ++k)
    if (!(wout[k] > wout[k - 1])) return fail(h, MROM_EINVAL, "mrom_adapt: omega_out must be strictly increasing");

  DevBuf Dbuf, Delta, snaps_d, lam_d, arg_d;
  e = cudaMalloc(&Dbuf.p, (size_t)3 * ns_cap * n * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&Delta.p, (size_t)n_out * 9 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&snaps_d.p, ns_cap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&lam_d.p, ns_cap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&arg_d.p, ns_cap * sizeof(int));
  if (e == cudaSuccess && D0)
    e = cudaMemcpyAsync(Dbuf.p, D0, (size_t)3 * ns0 * n * sizeof(double2), cudaMemcpyDefault, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_adapt: allocation");
  auto* Dcols = static_cast<double2*>(Dbuf.p);
  // without a callback the library solves the full-order snapshots itself (mrom_fom_solve)
  auto gpu_snapshots = [&](const double* w, int nw, double2* dst) -> mrom_status {
    for (int k0 = 0; k0 < nw; k0 += MROM_MAX_FOM_RHS / 3) {
      const int nk = std::min(nw - k0, MROM_MAX_FOM_RHS / 3);
      const mrom_status fs = fom_solve(h, fom, w + k0, nk, kAdaptSolveTol, kAdaptSolveMaxIter,
                                       dst + (size_t)3 * k0 * n, n, nullptr, nullptr);
      if (fs != MROM_OK) return fs;
    }
    return MROM_OK;
  };
  if (!D0) {
    const mrom_status fs = gpu_snapshots(omega0, ns0, Dcols);
    if (fs != MROM_OK) return fs;
  }
  std::vector<double2> stage;  // host staging for the callback's snapshots
  std::vector<double> snaps(omega0, omega0 + ns0);
  const double b_alpha = fom->alpha * fom->alpha * fom->alpha * fom->vol_B;

  int ns = ns0, k = 1;
  double Lam = std::numeric_limits<double>::infinity();
  int nh = 0;
  mrom_rom_t rom = nullptr;
  auto rebuild = [&]() -> mrom_status {
    if (rom) mrom_rom_free(rom);
    rom = nullptr;
    return mrom_project(h, fom, Dcols, n, 3 * ns, opts->tol_sigma, opts->r_max, nullptr, 0, &rom, nullptr, nullptr);
  };
  mrom_status s = rebuild();
  if (s != MROM_OK) return s;
  while (Lam / b_alpha > opts->tol_delta && k < opts->max_k) {
    ++k;
    // certificates of the current reduced model on the output grid (Algorithm 1)
    s = mrom_certificate(h, &rom, 1, omega_out, n_out, 0, static_cast<double*>(Delta.p));
    if (s == MROM_OK) s = mrom_synchronize(h);
    if (s != MROM_OK) {
      mrom_rom_free(rom);
      return s;
    }
    std::vector<double> sorted = snaps;
    std::sort(sorted.begin(), sorted.end());
    const int nint = ns - 1;
    std::vector<double> lam(nint);
    std::vector<int> arg(nint);
    e = cudaMemcpyAsync(snaps_d.p, sorted.data(), ns * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      interval_max_kernel<<<nint, 256, 0, st>>>(static_cast<double*>(Delta.p), omega_out, n_out,
                                                static_cast<double*>(snaps_d.p), ns, static_cast<double*>(lam_d.p),
                                                static_cast<int*>(arg_d.p));
      ++h->launches;
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(lam.data(), lam_d.p, nint * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(arg.data(), arg_d.p, nint * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      mrom_rom_free(rom);
      return cuda_fail(h, e, "mrom_adapt: interval maxima");
    }
    // Lambda = max_n Lambda_n
    Lam = -std::numeric_limits<double>::infinity();
    for (int i = 0; i < nint; ++i)
      if (arg[i] >= 0) Lam = std::max(Lam, lam[i]);
    if (lambda_hist && nh < opts->max_k) lambda_hist[nh] = Lam;
    ++nh;
    if (!(Lam / b_alpha > opts->tol_delta)) break;
    // the N* intervals with the largest Lambda_n, one new snapshot each; with a threshold,
    // only intervals with Lambda_n >= theta Lambda (still at most N* per iteration)
    std::vector<int> order(nint);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      const bool va = arg[a] >= 0, vb = arg[b] >= 0;
      if (va != vb) return va;
      return lam[a] > lam[b];
    });
    std::vector<double> fresh;
    for (int i = 0; i < nint && (int)fresh.size() < opts->n_star; ++i)
      if (arg[order[i]] >= 0 && (opts->theta <= 0.0 || lam[order[i]] >= opts->theta * Lam))
        fresh.push_back(wout[arg[order[i]]]);
    if (fresh.empty()) break;
    std::sort(fresh.begin(), fresh.end());
    const int nn = (int)fresh.size();
    // full-order snapshots from the caller, uploaded after the columns already held
    if (!cb) {
      const mrom_status fs = gpu_snapshots(fresh.data(), nn, Dcols + (size_t)3 * ns * n);
      if (fs != MROM_OK) {
        mrom_rom_free(rom);
        return fs;
      }
    } else {
      stage.assign((size_t)3 * nn * n, make_double2(0.0, 0.0));
      if (cb(user, nn, fresh.data(), stage.data()) != 0) {
        mrom_rom_free(rom);
        return fail(h, MROM_ECALLBACK, "mrom_adapt: snapshot callback returned an error");
      }
      e = cudaMemcpy(Dcols + (size_t)3 * ns * n, stage.data(), stage.size() * sizeof(double2), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        mrom_rom_free(rom);
        return cuda_fail(h, e, "mrom_adapt: snapshot upload");
      }
    }
    snaps.insert(snaps.end(), fresh.begin(), fresh.end());
    ns += nn;
    // updated TSVD and projection
    s = rebuild();
    if (s != MROM_OK) return s;
  }
  *out = rom;
  if (k_done) *k_done = k;
  if (ns_out) *ns_out = ns;
  if (omega_snap_out) {
    std::vector<double> sorted = snaps;
    std::sort(sorted.begin(), sorted.end());
    std::copy(sorted.begin(), sorted.end(), omega_snap_out);
  }
  return MROM_OK;
}
