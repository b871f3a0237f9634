// afn_device.cuh -- device helpers shared by the kernels of libafn.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace afn {

// Squared distance in FP64 summed over t = 0..d-1 in order with separately
// rounded multiply and add (no fused multiply-add), so that FPS and KNN
// decisions are reproducible bit for bit.
__device__ __forceinline__ double sqdist_exact(const double *x, const double *y, int d)
{
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
        double u = __dsub_rn(x[t], y[t]);
        s = __dadd_rn(s, __dmul_rn(u, u));
    }
    return s;
}

// Kernel value from a squared distance, FP64 (Gaussian eq. (gaussianf);
// Matern-3/2 of Sec. 5).  Written as the definition: exp(-r^2 / l^2) and
// (1 + sqrt3 r / l) exp(-sqrt3 r / l).
__device__ __forceinline__ double kernel64(double r2, int kernel, double l)
{
    if (kernel == 0) return exp(-(r2 / (l * l)));
    double r = sqrt(r2);
    double t = 1.7320508075688772 * r / l;
    return (1.0 + t) * exp(-t);
}

// FP32 fast path on pre-scaled points.
//   Gaussian: x~ = x sqrt(log2 e) / l   ->  K = 2^(-r~^2)
//   Matern:   x~ = x sqrt(3) / l        ->  t = r~, K = (1 + t) 2^(-t log2 e)
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int KER>
__device__ __forceinline__ float kernel32_scaled(float r2)
{
    if (KER == 0) return ex2_approx(-r2);
    float t = sqrt_approx(r2);
    return (1.0f + t) * ex2_approx(t * -1.4426950408889634f);
}

// Packed FP32 pairs (two floats in one 64-bit register, low = first):
// Blackwell's f32x2 add / sub / fma issue one instruction for two lanes of
// work.  Rounding is the same as the scalar .rn operations.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b)
{
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b)
{
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2_t f2_pack(float lo, float hi)
{
    f2_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}

__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// Lexicographic "better" for argmax with lowest-index tie-break.
__device__ __forceinline__ bool better_max(double v1, int64_t i1, double v2, int64_t i2)
{
    return (v1 > v2) || (v1 == v2 && i1 < i2);
}

__device__ __forceinline__ void warp_argmax(double &v, int64_t &i)
{
    for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int64_t i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (better_max(v2, i2, v, i)) { v = v2; i = i2; }
    }
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
// Sense via a generation counter.  Every wait is bounded: after
// `limit_ns` the waiting block sets *err = 2 and returns false; a block
// that sees *err set also stops waiting.  Returns true when every block
// arrived.
__device__ __forceinline__ bool grid_barrier(unsigned int *count, volatile unsigned int *gen,
                                             unsigned int nblocks, volatile int *err,
                                             uint64_t limit_ns)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned int g = *gen;
        __threadfence();
        unsigned int arrived = atomicAdd(count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd((unsigned int *)gen, 1u);
        } else {
            uint64_t t0 = globaltimer_ns();
            unsigned int spins = 0;
            while (*gen == g) {
                if (*err) { ok = 0; break; }
                if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > limit_ns) {
                    *err = 2;
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        ok_s = ok && (*err == 0);
    }
    __syncthreads();
    return ok_s != 0;
}

}  // namespace afn
