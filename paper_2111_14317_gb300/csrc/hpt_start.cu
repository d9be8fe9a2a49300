// Start points on the device: the |det V| solutions of the binomial start
// system of a pairs cell (Section 2: H(y, t = 0) = 0 keeps the cell's two
// monomials per equation), enumerated one thread per solution from the host's
// exact setup (binomial_setup: Hermite diagonal, adj V modulo |det V|).
// Solution `first + q` has the mixed-radix digits k (last coordinate
// fastest); its phase numerators are exact 64-bit modular sums (128-bit
// products).
#include <math.h>

#include "hpt_internal.h"

namespace hpt {
namespace {

__device__ __forceinline__ uint64_t mulmod(uint64_t a, uint64_t b, uint64_t L) {
  return (uint64_t)(((unsigned __int128)a * b) % L);
}

__global__ void __launch_bounds__(128) start_points_kernel(const __grid_constant__ StartConsts S, int64_t first,
                                                           int64_t count, double2* __restrict__ y0) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const int n = S.n;
  uint64_t k[kMaxN];
  int64_t idx = first + q;
  for (int j = n - 1; j >= 0; --j) {
    k[j] = (uint64_t)(idx % S.h[j]);
    idx /= S.h[j];
  }
  const double two_pi = 6.283185307179586476925286766559;
  for (int r = 0; r < n; ++r) {
    uint64_t num = 0;
    for (int j = 0; j < n; ++j)
      if (k[j]) num = (num + mulmod(S.adjm[r * n + j], k[j], S.D)) % S.D;   // below D < 2^62: no overflow
    const double frac = (double)num / (double)S.D;
    const double mag = exp(S.zr0[r]);
    double sn, cs;
    sincos(S.zi0[r] + two_pi * frac, &sn, &cs);
    y0[(size_t)q * n + r] = make_double2(mag * cs, mag * sn);
  }
}

}  // namespace
}  // namespace hpt

using namespace hpt;

extern "C" hpt_status hpt_binomial_start_device(int32_t n, const int32_t* msz, const int32_t* exps,
                                                const double* coeffs, const int32_t* pairs, int64_t first,
                                                int64_t count, void* y0_dev, int64_t* total, void* stream) {
  StartConsts S;
  hpt_status rc = binomial_setup(n, msz, exps, coeffs, pairs, first, count, y0_dev != nullptr, S, total);
  if (rc) return rc;
  if (count == 0) return HPT_OK;
  const int64_t blocks = (count + 127) / 128;
  if (blocks > 0x7fffffff) { set_error("count too large"); return HPT_ERANGE; }
  start_points_kernel<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(S, first, count, (double2*)y0_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HPT_OK : cuda_fail(e, "start point launch");
}
