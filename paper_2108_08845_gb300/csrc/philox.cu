// Gaussian test matrix of the randomized SVD (Sec. 3.3: a zero-mean,
// unit-variance Gaussian sketch, redrawn for every randomized SVD).
//
// Generator: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of
//   (hi0, lo0) = mulhilo(0xD2511F53, x0), (hi1, lo1) = mulhilo(0xCD9E8D57, x2),
//   x <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0),
// with the key bumped by (0x9E3779B9, 0xBB67AE85) between rounds.
// Variate idx of stream (seed, sid) uses counter (idx/2, idx/2 >> 32, sid,
// sid >> 32) and key (seed, seed >> 32).  Two 53-bit uniforms u1 in (0, 1]
// and u2 in [0, 1) feed Box-Muller (1958): r = sqrt(-2 ln u1), even idx ->
// r cos(2 pi u2), odd idx -> r sin(2 pi u2).
//
// ln and sin/cos are evaluated here from their series (atanh series of ln m
// after an exact binary exponent split; Taylor series of sin and cos on
// [0, pi/2) after an exact quadrant split of 4*u2) with every operation an
// explicitly rounded IEEE-754 binary64 intrinsic, so the variates are a fixed
// function of the Philox words, reproducible bit for bit by any
// implementation performing the same operations.  This file is compiled with
// -fmad=false as well.
#include "psvd_internal.cuh"

namespace psvd {
namespace {

__device__ __forceinline__ void philox4x32_10(uint32_t x[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * x[0], hi0 = __umulhi(0xD2511F53u, x[0]);
    const uint32_t lo1 = 0xCD9E8D57u * x[2], hi1 = __umulhi(0xCD9E8D57u, x[2]);
    const uint32_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
  }
}

// 1/(2k+1), k = 0..12
__constant__ double kAtanh[13] = {
    0x1p+0,                0x1.5555555555555p-2, 0x1.999999999999ap-3, 0x1.2492492492492p-3,
    0x1.c71c71c71c71cp-4,  0x1.745d1745d1746p-4, 0x1.3b13b13b13b14p-4, 0x1.1111111111111p-4,
    0x1.e1e1e1e1e1e1ep-5,  0x1.af286bca1af28p-5, 0x1.8618618618618p-5, 0x1.642c8590b2164p-5,
    0x1.47ae147ae147bp-5};
// (-1)^k/(2k+1)!, k = 0..12
__constant__ double kSin[13] = {
    0x1p+0,                 -0x1.5555555555555p-3, 0x1.1111111111111p-7,  -0x1.a01a01a01a01ap-13,
    0x1.71de3a556c734p-19,  -0x1.ae64567f544e4p-26, 0x1.6124613a86d09p-33, -0x1.ae7f3e733b81fp-41,
    0x1.952c77030ad4ap-49,  -0x1.2f49b46814157p-57, 0x1.71b8ef6dcf572p-66, -0x1.761b41316381ap-75,
    0x1.3f3ccdd165fa9p-84};
// (-1)^k/(2k)!, k = 0..12
__constant__ double kCos[13] = {
    0x1p+0,                -0x1p-1,                0x1.5555555555555p-5,  -0x1.6c16c16c16c17p-10,
    0x1.a01a01a01a01ap-16, -0x1.27e4fb7789f5cp-22, 0x1.1eed8eff8d898p-29, -0x1.93974a8c07c9dp-37,
    0x1.ae7f3e733b81fp-45, -0x1.6827863b97d97p-53, 0x1.e542ba4020225p-62, -0x1.0ce396db7f853p-70,
    0x1.f2cf01972f578p-80};

__device__ __forceinline__ double ln_series(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  long long e = (long long)((bits >> 52) & 0x7ffull) - 1023;
  double m = __longlong_as_double((long long)((bits & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
  if (m > 0x1.6a09e667f3bcdp+0) {  // 2 * sqrt(1/2) rounded: m in (sqrt 2, 2) -> halve
    m = __dmul_rn(m, 0.5);
    e += 1;
  }
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double z = __dmul_rn(s, s);
  double p = kAtanh[12];
#pragma unroll
  for (int k = 11; k >= 0; --k) p = __fma_rn(p, z, kAtanh[k]);
  const double lnm = __dmul_rn(__dmul_rn(2.0, s), p);
  return __fma_rn((double)e, 0x1.62e42fefa39efp-1, lnm);
}

__device__ __forceinline__ void sincos_2pi_series(double u, double* sn, double* cs) {
  const double u4 = __dmul_rn(4.0, u);
  const double qd = floor(u4);
  const int q = (int)qd;
  const double phi = __dmul_rn(__dsub_rn(u4, qd), 0x1.921fb54442d18p+0);
  const double z = __dmul_rn(phi, phi);
  double ps = kSin[12], pc = kCos[12];
#pragma unroll
  for (int k = 11; k >= 0; --k) {
    ps = __fma_rn(ps, z, kSin[k]);
    pc = __fma_rn(pc, z, kCos[k]);
  }
  const double s = __dmul_rn(phi, ps), c = pc;
  switch (q & 3) {
    case 0: *sn = s; *cs = c; break;
    case 1: *sn = c; *cs = -s; break;
    case 2: *sn = -s; *cs = -c; break;
    default: *sn = -c; *cs = s; break;
  }
}

__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
  const unsigned long long v = ((unsigned long long)(a >> 5) << 26) | (unsigned long long)(b >> 6);
  return __dmul_rn((double)v, 0x1p-53);
}

__device__ double gaussian_variate(uint64_t seed, uint64_t sid, uint64_t idx) {
  const uint64_t pair = idx >> 1;
  uint32_t x[4] = {(uint32_t)pair, (uint32_t)(pair >> 32), (uint32_t)sid, (uint32_t)(sid >> 32)};
  philox4x32_10(x, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = __dsub_rn(1.0, uniform53(x[0], x[1]));
  const double u2 = uniform53(x[2], x[3]);
  const double r = __dsqrt_rn(__dmul_rn(-2.0, ln_series(u1)));
  double sn, cs;
  sincos_2pi_series(u2, &sn, &cs);
  return (idx & 1) ? __dmul_rn(r, sn) : __dmul_rn(r, cs);
}

__global__ void gaussian_sketch_kernel(uint64_t seed, uint64_t sid, int64_t count,
                                       float* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    out[i] = __double2float_rn(gaussian_variate(seed, sid, (uint64_t)i));
}

}  // namespace

cudaError_t gaussian_sketch_launch(uint64_t seed, uint64_t stream_id, int64_t rows, int64_t cols,
                                   float* out, cudaStream_t st) {
  const int64_t count = rows * cols;
  if (count <= 0) return cudaSuccess;
  int64_t blocks = ceil_div(count, 256);
  if (blocks > 4096) blocks = 4096;
  gaussian_sketch_kernel<<<(unsigned)blocks, 256, 0, st>>>(seed, stream_id, count, out);
  return cudaGetLastError();
}

}  // namespace psvd
