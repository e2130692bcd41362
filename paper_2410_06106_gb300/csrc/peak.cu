// Measured FP32 FMA throughput, SM clock and shared-memory load bandwidth of the
// current GPU: the denominators of the operators' rooflines. The projector and
// the backprojector evaluate the system matrix on the fly (two saturating
// trapezoid FMAs and one accumulating FMA per touched bin) from data staged in
// shared memory, so their ceilings are the FP32 pipe and shared memory, not HBM.
//
// Every thread runs kPeakChains independent chains of dependent FMAs
// a <- a * b + c (b, c kernel arguments, so nothing folds), kPeakUnroll per loop
// trip, in scalar form (fmaf) and in packed form (__ffma2_rn, two FP32 lanes
// per instruction); the grid fills every SM at the occupancy the API reports.
// One thread also reads the SM cycle counter and the global nanosecond timer
// at its start and end, which gives the SM clock the kernel ran at. Both
// operators read two FP32 values of shared memory per update (the staged image
// band or the staged residual window), so the shared-memory bandwidth bounds
// them too; its microbenchmark is below.
#include "tomo_internal.cuh"

namespace tomo {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;

__device__ unsigned long long g_peak_clock[2];  // SM cycles, nanoseconds of block 0's thread 0
__device__ float g_peak_sink;                   // written only if the chains reach -1 (never)

__device__ __forceinline__ unsigned long long ns_timer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(int trips, float b, float c) {
    const unsigned long long t0 = ns_timer();
    const long long c0 = clock64();
    float s = 0.f;
    if constexpr (PACKED) {
        float2 a[kPeakChains];
        const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) a[k] = make_float2(1e-3f * threadIdx.x + k, 0.5f + k);
        for (int t = 0; t < trips; ++t) {
#pragma unroll
            for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
                for (int k = 0; k < kPeakChains; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
            }
        }
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) s += a[k].x + a[k].y;
    } else {
        float a[kPeakChains];
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) a[k] = 1e-3f * threadIdx.x + k;
        for (int t = 0; t < trips; ++t) {
#pragma unroll
            for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
                for (int k = 0; k < kPeakChains; ++k) a[k] = fmaf(a[k], b, c);
            }
        }
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) s += a[k];
    }
    if (s == -1.0f) g_peak_sink = s;  // the chains converge to c / (1 - b) > 0
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        g_peak_clock[0] = (unsigned long long)(clock64() - c0);
        g_peak_clock[1] = ns_timer() - t0;
    }
}

// Shared-memory load bandwidth: every thread reads 8 float2 per loop trip at
// addresses where a warp's 32 lanes cover 256 consecutive bytes (conflict-free:
// two wavefronts per warp load, the layout the backprojector's window loads
// have), moving through a 16 KB buffer so that no load can be hoisted out of
// the loop, into 8 independent accumulators.
constexpr int kSmemWords = kPeakThreads * 8;  // float2 entries of the buffer

__global__ void __launch_bounds__(kPeakThreads) smem_peak_kernel(int trips) {
    __shared__ float2 buf[kSmemWords];
    const int tid = threadIdx.x;
    for (int i = tid; i < kSmemWords; i += kPeakThreads) buf[i] = make_float2((float)i, 1.0f);
    __syncthreads();
    const unsigned base = (unsigned)__cvta_generic_to_shared(buf);
    float2 acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = make_float2(0.f, 0.f);
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const unsigned a = base + (unsigned)(((u * kPeakThreads + tid) + t * 32) & (kSmemWords - 1)) * 8u;
            float x, y;
            asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(x), "=f"(y) : "r"(a));
            acc[u].x += x;
            acc[u].y += y;
        }
    }
    float sum = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) sum += acc[u].x + acc[u].y;
    if (sum == -1.0f) g_peak_sink = sum;  // never: every value is >= 0
}

double run_smem_peak(int target_ms, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    TOMO_CUDA(cudaGetDevice(&dev));
    TOMO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TOMO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smem_peak_kernel, kPeakThreads, 0));
    const int blocks = sms * std::max(per_sm, 1);
    const double bytes_per_trip = 8.0 * sizeof(float2) * (double)blocks * kPeakThreads;
    cudaEvent_t e0, e1;
    TOMO_CUDA(cudaEventCreate(&e0));
    TOMO_CUDA(cudaEventCreate(&e1));
    auto timed = [&](int trips) {
        TOMO_CUDA(cudaEventRecord(e0, st));
        smem_peak_kernel<<<blocks, kPeakThreads, 0, st>>>(trips);
        TOMO_CUDA(cudaGetLastError());
        TOMO_CUDA(cudaEventRecord(e1, st));
        TOMO_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        TOMO_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return (double)ms;
    };
    int trips = 64;
    timed(trips);
    double ms = timed(trips);
    trips = (int)std::min(16777216.0, std::max(64.0, trips * target_ms / std::max(ms, 1e-3)));
    timed(trips);
    ms = timed(trips);
    TOMO_CUDA(cudaEventDestroy(e0));
    TOMO_CUDA(cudaEventDestroy(e1));
    return bytes_per_trip * trips / (ms * 1e-3) / 1e9;
}

struct PeakRun {
    double tflops;
    double mhz;
};

template <bool PACKED>
PeakRun run_peak(int target_ms, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    TOMO_CUDA(cudaGetDevice(&dev));
    TOMO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TOMO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<PACKED>, kPeakThreads, 0));
    const int blocks = sms * std::max(per_sm, 1);
    const double flop_per_trip =
        2.0 * (PACKED ? 2 : 1) * kPeakChains * kPeakUnroll * (double)blocks * kPeakThreads;
    const float b = 0.5f, c = 1.0f;
    cudaEvent_t e0, e1;
    TOMO_CUDA(cudaEventCreate(&e0));
    TOMO_CUDA(cudaEventCreate(&e1));
    auto timed = [&](int trips) {
        TOMO_CUDA(cudaEventRecord(e0, st));
        fma_peak_kernel<PACKED><<<blocks, kPeakThreads, 0, st>>>(trips, b, c);
        TOMO_CUDA(cudaGetLastError());
        TOMO_CUDA(cudaEventRecord(e1, st));
        TOMO_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        TOMO_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return (double)ms;
    };
    int trips = 64;
    timed(trips);  // warm-up (module load, clocks)
    double ms = timed(trips);
    // size the timed launch to about target_ms (at most 2^24 trips)
    trips = (int)std::min(16777216.0, std::max(64.0, trips * target_ms / std::max(ms, 1e-3)));
    timed(trips);
    ms = timed(trips);
    unsigned long long clk[2] = {0, 0};
    TOMO_CUDA(cudaMemcpyFromSymbol(clk, g_peak_clock, sizeof(clk)));
    TOMO_CUDA(cudaEventDestroy(e0));
    TOMO_CUDA(cudaEventDestroy(e1));
    PeakRun r;
    r.tflops = flop_per_trip * trips / (ms * 1e-3) / 1e12;
    r.mhz = clk[1] ? 1e3 * (double)clk[0] / (double)clk[1] : 0.0;
    return r;
}

}  // namespace
}  // namespace tomo

using namespace tomo;

extern "C" {

tomo_status tomo_fp32_peak(int target_ms, double* tflops_scalar, double* tflops_packed, double* sm_mhz,
                           tomo_stream_t stream) {
    return guard([&] {
        TOMO_REQUIRE(target_ms >= 1 && target_ms <= 2000, "target_ms must be in [1, 2000]");
        cudaStream_t st = (cudaStream_t)stream;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        TOMO_CUDA(cudaStreamIsCapturing(st, &cap));
        TOMO_REQUIRE(cap == cudaStreamCaptureStatusNone, "tomo_fp32_peak synchronizes: not on a capturing stream");
        const PeakRun s = run_peak<false>(target_ms, st);
        const PeakRun p = run_peak<true>(target_ms, st);
        if (tflops_scalar) *tflops_scalar = s.tflops;
        if (tflops_packed) *tflops_packed = p.tflops;
        if (sm_mhz) *sm_mhz = s.mhz;
    });
}

tomo_status tomo_smem_peak(int target_ms, double* gbs, tomo_stream_t stream) {
    return guard([&] {
        TOMO_REQUIRE(target_ms >= 1 && target_ms <= 2000, "target_ms must be in [1, 2000]");
        TOMO_REQUIRE(gbs, "gbs must be non-NULL");
        cudaStream_t st = (cudaStream_t)stream;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        TOMO_CUDA(cudaStreamIsCapturing(st, &cap));
        TOMO_REQUIRE(cap == cudaStreamCaptureStatusNone, "tomo_smem_peak synchronizes: not on a capturing stream");
        *gbs = run_smem_peak(target_ms, st);
    });
}

}  // extern "C"
