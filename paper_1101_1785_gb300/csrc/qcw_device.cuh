// Device helpers shared by the qcw CUDA kernels: complex64 arithmetic on float2 and
// label bit manipulation.
//
// Flat index of rho element (r, c) is g = r * 2^n + c, a 2n-bit number.  Its bits are the
// "virtual bits" of the kernels: bit (n-1-q) is qubit q's column bit and bit (2n-1-q) its
// row bit (qubit q has stride 2^(n-1-q) in a label, Sec. 2.3 Eq. staten).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qcw {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// acc += a * b
__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b)
{
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(float2 &acc, float2 a, float2 b)
{
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Insert a zero bit at position p of x (bits >= p move up by one).
__device__ __forceinline__ uint64_t insert0(uint64_t x, int p)
{
    uint64_t lo = x & ((1ull << p) - 1ull);
    return ((x ^ lo) << 1) | lo;
}

// Scatter the low bits of x onto positions pos[0..nb-1] (pos[j] receives bit j).
__device__ __forceinline__ uint64_t deposit(uint64_t x, const int8_t *pos, int nb)
{
    uint64_t r = 0;
    for (int j = 0; j < nb; j++) r |= ((x >> j) & 1ull) << pos[j];
    return r;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace qcw
