// probe.cu -- measured FP32 instruction rates of the current GPU.
//
// The c-transform and C-bar passes are bound by FP32 arithmetic on the CUDA
// cores (no dense contraction, no tensor cores), so their rooflines need the
// rate at which this GPU retires the instructions they use.  Each probe runs
// one instruction stream per thread: eight independent dependency chains,
// unrolled sixteen times per loop trip, on SMs x ctas_per_sm CTAs of 256
// threads (one wave: every CTA is resident from the start).  Rates are
// counted in FP32 results (a packed f32x2 instruction counts two; the
// c-transform mixes count candidates, i.e. (input, output) pairs) per clock
// per SM, from the SM cycle counter, and per second over the device, from
// CUDA events.  Not a step of the paper: a measurement of the hardware the
// passes are measured against.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <vector>

#include "common.cuh"

namespace qwb {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 16;

__device__ __forceinline__ float p_fma(float a, float b, float c) {
    float d;
    asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float p_sub_rm(float a, float b) {
    float d;
    asm("sub.rm.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float p_min2(float a, float b) {
    float d;
    asm("min.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float p_min3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ unsigned long long p_fma2(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long p_sub2_rm(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long p_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void p_unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// FP32 results per chain step of each kind (0..9)
__host__ __device__ constexpr int probe_results_per_step(int kind) {
    return (kind >= 4) ? 2 : 1;
}

// kinds 8, 9: the shifted line-paired c-transform's inner block in isolation
// (16 outputs per thread, chunks of 8 columns, the 23 squared column offsets
// in registers, two packed potentials per 16-byte shared load, one rounded-up
// packed subtraction per column, then per output one packed round-down
// subtraction and one 3-input min); 8 with each subtraction-and-min pair in
// one assembly block, 9 with separate blocks.  A chain step is one
// (column, output) candidate pair.
template <bool FUSED>
__device__ __forceinline__ void probe_ct_block(int iters, const ulonglong2* hs, float (&mins)[16]) {
    unsigned long long DD[23];
#pragma unroll
    for (int e = 0; e < 23; ++e) {
        const float d = (float)(e - 15 + (int)(threadIdx.x & 7));
        DD[e] = p_pack(d * d, d * d);
    }
    unsigned long long AA = p_pack(1.0f, 4.0f);
    for (int it = 0; it < iters; ++it) {
        const ulonglong2* hrow = hs + (it & 7) * 4;
#pragma unroll
        for (int s = 0; s < 8; s += 2) {
            const ulonglong2 v = hrow[s / 2];
            unsigned long long hA0, hA1;
            asm("sub.rp.f32x2 %0, %1, %2;" : "=l"(hA0) : "l"(v.x), "l"(AA));
            asm("sub.rp.f32x2 %0, %1, %2;" : "=l"(hA1) : "l"(v.y), "l"(AA));
#pragma unroll
            for (int ss = 0; ss < 2; ++ss) {
                const unsigned long long hA = ss ? hA1 : hA0;
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    if (FUSED) {
                        float d;
                        asm("{\n .reg .b64 t;\n .reg .f32 lo, hi;\n sub.rm.f32x2 t, %1, %2;\n mov.b64 {lo, hi}, t;\n"
                            " min.f32 %0, %3, lo, hi;\n}" : "=f"(d) : "l"(DD[s + ss - r + 15]), "l"(hA), "f"(mins[r]));
                        mins[r] = d;
                    } else {
                        const unsigned long long t = p_sub2_rm(DD[s + ss - r + 15], hA);
                        float lo, hi;
                        p_unpack(t, lo, hi);
                        mins[r] = p_min3(mins[r], lo, hi);
                    }
                }
            }
        }
        AA = p_pack(1.0f + (float)(it & 1), 4.0f);
    }
}

// kind: 0 fma.rn.f32, 1 sub.rm.f32, 2 min.f32 (2 inputs), 3 min.f32 (3 inputs),
// 4 fma.rn.f32x2, 5 sub.rm.f32x2, 6 sub.rm.f32x2 + 3-input min (two candidates),
// 7 two sub.rm.f32 + 3-input min (two candidates).  The chains stay finite:
// the subtrahend and addend are tiny, the multiplier just below one.
template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS, 2)
probe_ct_kernel(int iters, float seed, float* __restrict__ sink, long long* __restrict__ cycles) {
    __shared__ ulonglong2 hs[64];
    if (threadIdx.x < 64) {
        const float a = seed + (float)threadIdx.x, b = seed - (float)threadIdx.x;
        hs[threadIdx.x] = make_ulonglong2(p_pack(a, b), p_pack(b, a));
    }
    float mins[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) mins[r] = 1e30f;
    __syncthreads();
    long long t0 = clock64();
    probe_ct_block<KIND == 8>(iters, hs, mins);
    __syncthreads();
    long long t1 = clock64();
    float acc = 0.0f;
#pragma unroll
    for (int r = 0; r < 16; ++r) acc += mins[r];
    if (acc == 1234.5f) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        cycles[3 * blockIdx.x] = t0;
        cycles[3 * blockIdx.x + 1] = t1;
        cycles[3 * blockIdx.x + 2] = (long long)smid;
    }
}

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS)
probe_kernel(int iters, float seed, float* __restrict__ sink, long long* __restrict__ cycles) {
    float x[PROBE_CHAINS], y[PROBE_CHAINS], z[PROBE_CHAINS];
    unsigned long long xp[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) {
        x[k] = seed + 0.125f * k + 1e-3f * (float)threadIdx.x;
        y[k] = x[k] + 0.5f;
        z[k] = x[k] + 0.25f;
        xp[k] = p_pack(x[k], y[k]);
    }
    const float a = 0.99999994f, c = 1e-30f;
    const unsigned long long a2 = p_pack(a, a), c2 = p_pack(c, c);
    __syncthreads();
    long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) {
                if constexpr (KIND == 0) {
                    x[k] = p_fma(x[k], a, c);
                } else if constexpr (KIND == 1) {
                    x[k] = p_sub_rm(x[k], c);
                } else if constexpr (KIND == 2) {
                    x[k] = p_min2(x[k], x[(k + 1) % PROBE_CHAINS]);          // chains coupled cyclically
                } else if constexpr (KIND == 3) {
                    x[k] = p_min3(x[k], x[(k + 1) % PROBE_CHAINS], x[(k + 2) % PROBE_CHAINS]);
                } else if constexpr (KIND == 4) {
                    xp[k] = p_fma2(xp[k], a2, c2);
                } else if constexpr (KIND == 5) {
                    xp[k] = p_sub2_rm(xp[k], c2);
                } else if constexpr (KIND == 6) {
                    xp[k] = p_sub2_rm(xp[k], c2);
                    float lo, hi;
                    p_unpack(xp[k], lo, hi);
                    y[k] = p_min3(y[k], lo, hi);
                } else {
                    x[k] = p_sub_rm(x[k], c);
                    z[k] = p_sub_rm(z[k], c);
                    y[k] = p_min3(y[k], x[k], z[k]);
                }
            }
        }
    }
    __syncthreads();
    long long t1 = clock64();
    float acc = 0.0f;                 // only the chains this kind advanced stay live
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) {
        float lo, hi;
        p_unpack(xp[k], lo, hi);
        if constexpr (KIND <= 3) acc += x[k];
        else if constexpr (KIND <= 5) acc += lo + hi;
        else if constexpr (KIND == 6) acc += lo + hi + y[k];
        else acc += x[k] + y[k] + z[k];
    }
    if (acc == 1234.5f) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;   // keeps the chains live
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        cycles[3 * blockIdx.x] = t0;
        cycles[3 * blockIdx.x + 1] = t1;
        cycles[3 * blockIdx.x + 2] = (long long)smid;
    }
}

template <int KIND>
int probe_launch(int grid, int iters, float* sink, long long* cycles, cudaStream_t s) {
    if constexpr (KIND >= 8) probe_ct_kernel<KIND><<<grid, PROBE_THREADS, 0, s>>>(iters, 1.0f, sink, cycles);
    else probe_kernel<KIND><<<grid, PROBE_THREADS, 0, s>>>(iters, 1.0f, sink, cycles);
    QWB_LAUNCHED();
    return QWB_OK;
}

const void* probe_kernel_for(int kind) {
    switch (kind) {
        case 0: return (const void*)probe_kernel<0>;
        case 1: return (const void*)probe_kernel<1>;
        case 2: return (const void*)probe_kernel<2>;
        case 3: return (const void*)probe_kernel<3>;
        case 4: return (const void*)probe_kernel<4>;
        case 5: return (const void*)probe_kernel<5>;
        case 6: return (const void*)probe_kernel<6>;
        case 7: return (const void*)probe_kernel<7>;
        case 8: return (const void*)probe_ct_kernel<8>;
        default: return (const void*)probe_ct_kernel<9>;
    }
}

int probe_dispatch(int kind, int grid, int iters, float* sink, long long* cycles, cudaStream_t s) {
    switch (kind) {
        case 0: return probe_launch<0>(grid, iters, sink, cycles, s);
        case 1: return probe_launch<1>(grid, iters, sink, cycles, s);
        case 2: return probe_launch<2>(grid, iters, sink, cycles, s);
        case 3: return probe_launch<3>(grid, iters, sink, cycles, s);
        case 4: return probe_launch<4>(grid, iters, sink, cycles, s);
        case 5: return probe_launch<5>(grid, iters, sink, cycles, s);
        case 6: return probe_launch<6>(grid, iters, sink, cycles, s);
        case 7: return probe_launch<7>(grid, iters, sink, cycles, s);
        case 8: return probe_launch<8>(grid, iters, sink, cycles, s);
        case 9: return probe_launch<9>(grid, iters, sink, cycles, s);
        default: return QWB_ERR_INVALID_ARG;
    }
}

}  // namespace
}  // namespace qwb

using namespace qwb;

extern "C" int qwb_probe_fp32_rate(int32_t kind, int32_t ctas_per_sm, int32_t iters, double* out_h) {
    if (kind < 0 || kind > 9 || ctas_per_sm < 1 || ctas_per_sm > 8 || iters < 1 || !out_h) {
        set_last_error("qwb_probe_fp32_rate: kind in [0, 9], ctas_per_sm in [1, 8], iters >= 1, out_h non-null");
        return QWB_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    QWB_CUDA(cudaGetDevice(&dev));
    QWB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // one wave: no more CTAs per SM than can be resident at once
    int occ = 1;
    QWB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, probe_kernel_for(kind), PROBE_THREADS, 0));
    ctas_per_sm = std::max(1, std::min(ctas_per_sm, occ));
    const int grid = sms * ctas_per_sm;
    float* sink = nullptr;
    long long* cycles = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = QWB_OK;
    std::vector<long long> cyc(3 * (size_t)grid);
    float ms = 0.0f;
    auto cleanup = [&]() {
        if (sink) cudaFree(sink);
        if (cycles) cudaFree(cycles);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
#define PROBE_TRY(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) { cleanup(); return cuda_fail(e_, #call); } \
    } while (0)
    PROBE_TRY(cudaMalloc(&sink, sizeof(float) * (size_t)grid * PROBE_THREADS));
    PROBE_TRY(cudaMalloc(&cycles, sizeof(long long) * 3 * (size_t)grid));
    PROBE_TRY(cudaEventCreate(&e0));
    PROBE_TRY(cudaEventCreate(&e1));
    cudaStream_t s = 0;
    // warm-up (module load, clocks up), then the timed run
    if ((st = probe_dispatch(kind, grid, std::max(1, iters / 8), sink, cycles, s))) { cleanup(); return st; }
    PROBE_TRY(cudaEventRecord(e0, s));
    if ((st = probe_dispatch(kind, grid, iters, sink, cycles, s))) { cleanup(); return st; }
    PROBE_TRY(cudaEventRecord(e1, s));
    PROBE_TRY(cudaEventSynchronize(e1));
    PROBE_TRY(cudaEventElapsedTime(&ms, e0, e1));
    PROBE_TRY(cudaMemcpy(cyc.data(), cycles, sizeof(long long) * 3 * (size_t)grid, cudaMemcpyDeviceToHost));
#undef PROBE_TRY
    cleanup();
    // per SM: the span of its cycle counter from the first CTA's start to the
    // last CTA's end, and the CTAs it ran (CTAs need not all be co-resident)
    int max_sm = 0;
    for (int i = 0; i < grid; ++i) max_sm = std::max(max_sm, (int)cyc[3 * (size_t)i + 2]);
    std::vector<long long> lo(max_sm + 1, LLONG_MAX), hi(max_sm + 1, LLONG_MIN);
    std::vector<int> cnt(max_sm + 1, 0);
    for (int i = 0; i < grid; ++i) {
        const int sm = (int)cyc[3 * (size_t)i + 2];
        lo[sm] = std::min(lo[sm], cyc[3 * (size_t)i]);
        hi[sm] = std::max(hi[sm], cyc[3 * (size_t)i + 1]);
        cnt[sm]++;
    }
    double span_sum = 0.0;
    int used = 0, most = 0;
    for (int sm = 0; sm <= max_sm; ++sm)
        if (cnt[sm]) { span_sum += (double)(hi[sm] - lo[sm]); ++used; most = std::max(most, cnt[sm]); }
    const double per_cta = (double)PROBE_THREADS * iters * PROBE_UNROLL * PROBE_CHAINS *
                           probe_results_per_step(kind);
    out_h[0] = per_cta * grid / span_sum;                        // results per cycle per SM
    out_h[1] = per_cta * grid / (ms * 1e-3);                     // results per second, whole device
    out_h[2] = span_sum / used / (ms * 1e-3) / 1e6;              // cycle-counter MHz over the run
    out_h[3] = (double)sms;
    out_h[4] = (double)ctas_per_sm;
    out_h[5] = (double)most;                                     // most CTAs one SM ran
    return QWB_OK;
}
