// Rotation-invariant features of the spectral signature (Sect. 1): under a rotation Q of the
// object each coefficient matrix becomes Q M Q^T, so the eigenvalues of R~ = N0 + R and of I
// at each frequency are orientation independent and serve for dictionary matching.  One
// thread per matrix: the eigenvalues of its symmetric part in ascending order by sym3_eig
// (eig3.cuh: the trigonometric solution for the outermost eigenvalue, deflation and a closed-form
// 2 x 2 problem; a few eps ||M||, repeated eigenvalues included).  The sweep computes the same
// invariants in its epilogue (mrom_plan_sweep_invariants); this kernel serves stored outputs.
#include "mrom_internal.h"
#include "eig3.cuh"

namespace mrom {
namespace {

__global__ void eig3_kernel(const double* __restrict__ M, int64_t n, double* __restrict__ eig) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double* m = M + t * 9;
    sym3_eig(m[0], m[4], m[8], 0.5 * (m[1] + m[3]), 0.5 * (m[2] + m[6]), 0.5 * (m[5] + m[7]), eig[t * 3 + 0],
             eig[t * 3 + 1], eig[t * 3 + 2]);
  }
}

}  // namespace
}  // namespace mrom

using namespace mrom;

extern "C" mrom_status mrom_invariants(mrom_handle h, const double* M, int64_t n, double* eig) {
  if (!h) return MROM_EINVAL;
  if (n < 0 || (n > 0 && (!M || !eig))) return fail(h, MROM_EINVAL, "mrom_invariants: bad arguments");
  if (n == 0) return MROM_OK;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_invariants: cudaSetDevice");
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 65535LL * 8);
  eig3_kernel<<<(unsigned)blocks, 256, 0, h->stream>>>(M, n, eig);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_invariants: launch");
  ++h->launches;
  return MROM_OK;
}
