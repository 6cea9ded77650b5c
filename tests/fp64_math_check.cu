// Accuracy of the library's FP64 Newton-Raphson reciprocal, quotient and
// inverse cube root (swe_kernels.cuh) against CUDA's IEEE division and cbrt,
// over 2^20 seeded arguments log-uniform in [2^-30, 2^30]. Prints the largest
// error of each in units of the last place of the IEEE result. Test code:
// built and run by tests/test_gpu_fp64_math.py.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "../paper_1807_00672_gb300/csrc/swe_kernels.cuh"

__global__ void k_check(const double* x, const double* y, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = x[i], b = y[i];
  const double r = 1.0 / a, q = b / a, c = 1.0 / cbrt(a);
  const double ulp_r = fabs(r) * 2.220446049250313e-16;
  const double ulp_q = fabs(q) * 2.220446049250313e-16;
  const double ulp_c = fabs(c) * 2.220446049250313e-16;
  out[3 * i + 0] = fabs(swe::rcp_nr(a) - r) / ulp_r;
  out[3 * i + 1] = fabs(swe::Ops<double>::div(b, a) - q) / ulp_q;
  out[3 * i + 2] = fabs(swe::icbrt_nr(a) - c) / ulp_c;
}

int main() {
  const int n = 1 << 20;
  double* hx = new double[n];
  double* hy = new double[n];
  uint64_t s = 0x9E3779B97F4A7C15ull;
  auto next = [&]() {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    return (double)(s >> 11) / 9007199254740992.0;
  };
  for (int i = 0; i < n; ++i) {
    hx[i] = std::exp2(-30.0 + 60.0 * next());
    hy[i] = std::exp2(-30.0 + 60.0 * next()) * (next() < 0.5 ? -1.0 : 1.0);
  }
  double *dx, *dy, *dout;
  if (cudaMalloc(&dx, n * 8) != cudaSuccess || cudaMalloc(&dy, n * 8) != cudaSuccess ||
      cudaMalloc(&dout, 3 * (size_t)n * 8) != cudaSuccess) {
    printf("alloc failed\n");
    return 2;
  }
  cudaMemcpy(dx, hx, n * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dy, hy, n * 8, cudaMemcpyHostToDevice);
  k_check<<<(n + 255) / 256, 256>>>(dx, dy, n, dout);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    printf("kernel failed\n");
    return 3;
  }
  double* ho = new double[3 * (size_t)n];
  cudaMemcpy(ho, dout, 3 * (size_t)n * 8, cudaMemcpyDeviceToHost);
  double mx[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) mx[c] = std::fmax(mx[c], ho[3 * i + c]);
  printf("rcp %.3f\ndiv %.3f\nicbrt %.3f\n", mx[0], mx[1], mx[2]);
  return 0;
}
