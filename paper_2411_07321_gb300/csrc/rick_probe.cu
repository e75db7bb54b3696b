// rick_probe.cu -- measured per-SM throughput of the on-chip units that bound
// the gridding and transform kernels: shared-memory read-modify-writes (plain
// and atomic) and FP32 fused multiply-adds.  The bench divides each kernel's
// algorithmic work by these rates to state its shared-memory or arithmetic
// roofline, as it divides bytes by the measured HBM copy bandwidth.
//
// One CTA of 1024 threads per SM; each thread repeats an operation on eight
// words (or registers) of its own, so there are no bank conflicts and eight
// independent chains per thread.  Every CTA times its loop with clock64(), so
// the result is in operations per SM clock, independent of the clock speed.
#include <algorithm>
#include <vector>

#include "rick_common.cuh"

#define PROBE_THREADS 1024
#define PROBE_WORDS 8

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS, 1)
    probe_kernel(int iters, unsigned long long *cycles, float *sink)
{
    extern __shared__ __align__(16) unsigned long long s64[];  // PROBE_WORDS * PROBE_THREADS
    float *s32 = (float *)s64;
    unsigned int *u32 = (unsigned int *)s64;
    const int t = threadIdx.x;
#pragma unroll
    for (int j = 0; j < PROBE_WORDS; ++j) s64[t + PROBE_THREADS * j] = 0ull;
    __syncthreads();
    const float v = 1.0f + (float)t * 1e-7f;
    float acc = 0.0f;
    const unsigned long long c0 = clock64();
    if (KIND == RICK_PROBE_SMEM_RMW) {
        volatile float *vs = s32;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < PROBE_WORDS; ++j) vs[t + PROBE_THREADS * j] += v;
        }
    } else if (KIND == RICK_PROBE_SMEM_ATOMIC_F32) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < PROBE_WORDS; ++j) atomicAdd(&s32[t + PROBE_THREADS * j], v);
        }
    } else if (KIND == RICK_PROBE_SMEM_ATOMIC_U32) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < PROBE_WORDS; ++j) atomicAdd(&u32[t + PROBE_THREADS * j], 3u);
        }
    } else if (KIND == RICK_PROBE_SMEM_ATOMIC_U64) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < PROBE_WORDS; ++j) atomicAdd(&s64[t + PROBE_THREADS * j], 3ull);
        }
    } else if (KIND == RICK_PROBE_FFMA) {
        float r[PROBE_WORDS];
#pragma unroll
        for (int j = 0; j < PROBE_WORDS; ++j) r[j] = v + j;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < PROBE_WORDS; ++j) r[j] = __fmaf_rn(r[j], 0.999999f, 1e-7f);
        }
#pragma unroll
        for (int j = 0; j < PROBE_WORDS; ++j) acc += r[j];
    } else if (KIND == RICK_PROBE_FFMA2) {
        float2 r[PROBE_WORDS];
#pragma unroll
        for (int j = 0; j < PROBE_WORDS; ++j) r[j] = make_float2(v + j, v - j);
        const float2 a = make_float2(0.999999f, 0.999998f), b = make_float2(1e-7f, 2e-7f);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < PROBE_WORDS; ++j) r[j] = __ffma2_rn(r[j], a, b);
        }
#pragma unroll
        for (int j = 0; j < PROBE_WORDS; ++j) acc += r[j].x + r[j].y;
    } else if (KIND == RICK_PROBE_SHFL) {
        float r[PROBE_WORDS];
#pragma unroll
        for (int j = 0; j < PROBE_WORDS; ++j) r[j] = v + j;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < PROBE_WORDS; ++j)
                r[j] = __shfl_sync(0xffffffffu, r[j], (threadIdx.x + j + 1) & 31);
        }
#pragma unroll
        for (int j = 0; j < PROBE_WORDS; ++j) acc += r[j];
    } else if (KIND == RICK_PROBE_F2I) {
        // float to integer, round to nearest (cvt.rni.s32.f32), chained through
        // an integer add so that every conversion is live
        int r[PROBE_WORDS];
#pragma unroll
        for (int j = 0; j < PROBE_WORDS; ++j) r[j] = t + j;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < PROBE_WORDS; ++j) r[j] = __float2int_rn(__int_as_float(r[j] | 0x3f800000));
        }
#pragma unroll
        for (int j = 0; j < PROBE_WORDS; ++j) acc += (float)r[j];
    }
    __syncthreads();
    const unsigned long long c1 = clock64();
    if (t == 0) cycles[blockIdx.x] = c1 - c0;
    // keep the results observable
    sink[blockIdx.x * PROBE_THREADS + t] = acc + s32[t] + (float)u32[t + PROBE_THREADS];
}

template <int KIND>
static cudaError_t probe_launch(int blocks, int iters, unsigned long long *cyc, float *sink)
{
    const int smem = (int)(sizeof(unsigned long long) * PROBE_WORDS * PROBE_THREADS);
    cudaError_t e = cudaFuncSetAttribute(probe_kernel<KIND>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    probe_kernel<KIND><<<blocks, PROBE_THREADS, smem>>>(iters, cyc, sink);
    return cudaGetLastError();
}

extern "C" rick_status rick_probe_throughput(int32_t kind, double *ops_per_clock_per_sm)
{
    if (!ops_per_clock_per_sm || kind < RICK_PROBE_SMEM_RMW || kind > RICK_PROBE_F2I)
        return RICK_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RICK_ECUDA;
    unsigned long long *cyc = NULL;
    float *sink = NULL;
    if (cudaMalloc((void **)&cyc, sizeof(unsigned long long) * sms) != cudaSuccess)
        return RICK_ENOMEM;
    if (cudaMalloc((void **)&sink, sizeof(float) * (size_t)sms * PROBE_THREADS) != cudaSuccess) {
        cudaFree(cyc);
        return RICK_ENOMEM;
    }
    const int iters = (kind == RICK_PROBE_FFMA || kind == RICK_PROBE_FFMA2) ? 16384 : 2048;
    // (each conversion above also pays an OR: the figure bounds F2I from below)
    rick_status st = RICK_OK;
    std::vector<unsigned long long> h((size_t)sms);
    for (int rep = 0; rep < 2 && st == RICK_OK; ++rep) {  // the first run warms up
        cudaError_t e = cudaErrorInvalidValue;
        switch (kind) {
        case RICK_PROBE_SMEM_RMW: e = probe_launch<RICK_PROBE_SMEM_RMW>(sms, iters, cyc, sink); break;
        case RICK_PROBE_SMEM_ATOMIC_F32: e = probe_launch<RICK_PROBE_SMEM_ATOMIC_F32>(sms, iters, cyc, sink); break;
        case RICK_PROBE_SMEM_ATOMIC_U32: e = probe_launch<RICK_PROBE_SMEM_ATOMIC_U32>(sms, iters, cyc, sink); break;
        case RICK_PROBE_SMEM_ATOMIC_U64: e = probe_launch<RICK_PROBE_SMEM_ATOMIC_U64>(sms, iters, cyc, sink); break;
        case RICK_PROBE_FFMA: e = probe_launch<RICK_PROBE_FFMA>(sms, iters, cyc, sink); break;
        case RICK_PROBE_FFMA2: e = probe_launch<RICK_PROBE_FFMA2>(sms, iters, cyc, sink); break;
        case RICK_PROBE_SHFL: e = probe_launch<RICK_PROBE_SHFL>(sms, iters, cyc, sink); break;
        case RICK_PROBE_F2I: e = probe_launch<RICK_PROBE_F2I>(sms, iters, cyc, sink); break;
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess)
            e = cudaMemcpy(h.data(), cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = RICK_ECUDA;
    }
    cudaFree(cyc);
    cudaFree(sink);
    if (st != RICK_OK) return st;
    std::sort(h.begin(), h.end());
    const double c = (double)h[h.size() / 2];  // median over the SMs
    // FMAs count two per lane for the paired form
    const double per_op = (kind == RICK_PROBE_FFMA2) ? 2.0 : 1.0;
    *ops_per_clock_per_sm = c > 0.0 ? per_op * PROBE_THREADS * (double)iters * PROBE_WORDS / c : 0.0;
    return RICK_OK;
}
