// cmc_check_arith: the integer-pipe FP64 operations of the kernels (the
// correctly rounded product, quotient and square root built from 64-bit
// integer arithmetic in cmc_device.cuh) compared bit for bit with the FP64
// hardware operations on hashed operands, so that a test can confirm on
// the GPU itself that the replacements return the IEEE-754 results.
#include "cmc_device.cuh"
#include "../../include/cmc.h"

namespace {

using namespace cmc;

// splitmix64's output function (Steele, Lea and Flood 2014)
__device__ __forceinline__ unsigned long long hash64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// operand i of family f: 0 any bit pattern; 1 a random sign and
// significand with the exponent in 2^-40 .. 2^40; 2 as 1 with the low
// 0..52 significand bits cleared (exact results and ties)
__device__ __forceinline__ double operand(unsigned long long i, int f) {
  const unsigned long long x = hash64(i), y = hash64(i ^ 0x5DEECE66Dull);
  if (f == 0) return __longlong_as_double((long long)x);
  unsigned long long man = x & 0xFFFFFFFFFFFFFull;
  if (f == 2) man &= ~((1ull << (unsigned)(y % 53ull)) - 1ull);
  const unsigned long long ex = 983ull + (y >> 8) % 81ull;
  return __longlong_as_double((long long)(((y >> 63) << 63) | (ex << 52) | man));
}

__global__ void k_check_arith(int op, unsigned long long n, unsigned long long seed,
                              unsigned long long* bad) {
  unsigned long long mine = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int f = (int)(i % 3ull);
    const double a = operand(seed + 2 * i, f), b = operand(seed + 2 * i + 1, f);
    double hw, in;
    if (op == 0) { hw = __dmul_rn(a, b); in = mul_rn(a, b); }
    else if (op == 1) { hw = __ddiv_rn(a, b); in = div_rn(a, b); }
    else { hw = __dsqrt_rn(a); in = sqrt_rn(a); }
    const bool both_nan = hw != hw && in != in;
    if (ubits(hw) != ubits(in) && !both_nan) ++mine;
  }
  if (mine) atomicAdd(bad, mine);
}

}  // namespace

cmc_status cmc_check_arith(int32_t op, uint64_t n, uint64_t seed, uint64_t* mismatches) {
  if (op < 0 || op > 2 || !mismatches) return CMC_EINVAL;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) return CMC_ECUDA;
  cudaError_t e = cudaMemset(d, 0, sizeof(unsigned long long));
  if (!e && n) {
    k_check_arith<<<152 * 8, 256>>>(op, (unsigned long long)n, (unsigned long long)seed, d);
    e = cudaGetLastError();
  }
  unsigned long long h = 0;
  if (!e) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e) return CMC_ECUDA;
  *mismatches = (uint64_t)h;
  return CMC_OK;
}
