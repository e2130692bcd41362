// Message quantizers of dADMM-K and dADMM-J (Sec. 2.7) on GB300:
//   - scalar K-means (Algorithm 5): one CTA per vector, seeded initialisation
//     from probes staged in shared memory, FP32 nearest-centre decisions by
//     binary search over the sorted centres, exact 64-bit fixed-point centroid
//     sums in one shared slot per (centre, lane) added with 32-bit shared
//     atomics (integer sums: order-independent, so deterministic), means in FP64;
//   - JPEG-style codec: one thread per 8x8 block, the orthonormal DCT-II and
//     its inverse separable in registers on the FP32 cores, luminance table
//     of ITU-T T.81 Annex K scaled by the IJG quality rule.
// Both have a standalone entry (quant_kmeans / quant_jpeg) and a dADMM form
// that takes every owner segment of an iteration in one launch.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "tomo_internal.cuh"

namespace tomo {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;

// ------------------------------------------------------------------
// K-means
// ------------------------------------------------------------------
size_t kmeans_smem(int kmax) {
    return (size_t)2 * (kmax + 1) * 32 * sizeof(long long) + (kmax + 4) * sizeof(float) + 32 * sizeof(double);
}

// Nearest centre by FP32 distance |v - c_j| with ties to the lower index, over
// centres sorted ascending (s_cent, padded with +inf up to KMAX). The computed
// distance fl(v - c_j) of the centres at or below v falls (weakly) as j grows
// and fl(c_j - v) of those above v rises, because rounding is monotone; so
// with p = #{j : c_j <= v} (a branch-free binary search) the nearest centre is
// p - 1 or p, and among equal distances on the left the lowest index is found
// by walking down a run of equal values (only duplicate centres, or centres
// closer together than the rounding of v - c, make that run longer than 1).
// Without early exits: the search steps a pointer, and sentinels around the
// centres (s_cent[-2] = s_cent[-1] = -inf, s_cent[KMAX] = +inf) let the
// neighbours c[p - 2], c[p - 1] and c[p] load together without clamping. The
// result is final unless `walk` is set (the first step of the walk applies:
// duplicate or nearly equal centres); walk_down then finishes it from there.
template <int KMAX>
__device__ __forceinline__ int nearest_centre_flat(const float* s_cent, int k, float v, bool& walk, float& dl) {
    const float* c = s_cent;
#pragma unroll
    for (int step = KMAX / 2; step >= 1; step >>= 1) c += c[step - 1] <= v ? step : 0;
    c += c[0] <= v ? 1 : 0;
    const int p = min((int)(c - s_cent), k);  // the +inf padding counts only for v = +inf
    c = s_cent + p;
    const float cm2 = c[-2], cm1 = c[-1], cp = c[0];
    dl = v - cm1;
    const bool up = p < k && cp - v < dl;  // strict: a tie stays with the lower index
    const int best = p == 0 ? 0 : (up ? p : p - 1);
    walk = !up && best > 0 && v - cm2 == dl;
    return best;
}

// the rest of the walk, from a centre `best` whose lower neighbour is at the same distance dl
__device__ __forceinline__ int walk_down(const float* s_cent, int best, float v, float dl) {
    --best;
    while (best > 0 && v - s_cent[best - 1] == dl) --best;
    return best;
}

template <int KMAX>
__device__ void kmeans_block(const float* __restrict__ in, long long n, int k, int iters, uint64_t key,
                             uint8_t* codes, float* cent_out, float* deq, double* obj) {
    constexpr int NT = kKmThreads, NW = kKmThreads / 32;
    extern __shared__ __align__(16) unsigned char km_smem[];
    // member sums and counts: one slot per (centre, lane), shared by the block's warps
    // (shared-memory atomic adds; lanes of one warp never share a slot). Row KMAX takes
    // the adds of the positions past the end of a ragged last trip and is never read.
    // Shared memory has native 32-bit atomic adds only (64-bit adds are compare-and-swap
    // loops), so a fixed-point value q = hi 2^32 + a 2^16 + b (hi = q >> 32 signed, a
    // and b the two 16-bit halves of its low word) is added as three 32-bit pieces, with
    // a 32-bit count. A lane's slot takes at most min(n, n / 32 + 4) values per pass, so
    // the sums of a and b stay below 2^32 for n < 2^21 - 128, and that of hi
    // (|hi| < 2^(30 - lg n), at most n <= 2^lg n of them) below 2^30; longer inputs take
    // 64-bit slots added by compare-and-swap.
    constexpr int CNT = (KMAX + 1) * 32;  // words (or 64-bit slots) per array
    unsigned* s_w32 = reinterpret_cast<unsigned*>(km_smem);  // [4][KMAX + 1][32]: hi, a, b, count
    unsigned long long* s_sum = reinterpret_cast<unsigned long long*>(km_smem);  // [KMAX + 1][32], long inputs
    unsigned long long* s_cnt = s_sum + CNT;                                      // [KMAX + 1][32], long inputs
    float* s_cent = reinterpret_cast<float*>(s_sum + 2 * CNT) + 2;  // [-2, KMAX]: sentinels at -2, -1, KMAX
    // 32 doubles after the centres: byte offset 16 CNT + 4 (KMAX + 4), a multiple of 8
    double* s_red = reinterpret_cast<double*>(km_smem + (size_t)16 * CNT + 4 * (KMAX + 4));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned full = 0xffffffffu;
    const uint64_t un = (uint64_t)n;
    const bool split = n < (1ll << 21) - 128;  // 32-bit pieces of the member sums (below)
    // 16-byte loads and stores when the segment and the output allow them (uniform per block)
    const bool vec = (n & 3) == 0 && ((uintptr_t)in & 15) == 0 && ((uintptr_t)deq & 15) == 0;

    // Member sums are exact 64-bit fixed-point sums, scale 2^sh with
    // |v| 2^sh < 2^(62 - lg n) for every value, so that n of them fit: exact and
    // independent of the summation order. The scaled value v 2^sh is exact in
    // FP32 (a power-of-two scale); only its fraction below 2^0, i.e. below
    // 2^(lg n - 62) max|v|, is rounded away.
    //
    // Initial centres: value at a seeded index, moving to the next index while
    // the value is already a centre (64 probes at most, checked 32 at a time).
    // Every block thread first loads the probes of every centre (they are in
    // flight during the max|v| pass and stored to the member-sum slots, free
    // until the first iteration, after it), so that the sequential choice below
    // reads only shared memory.
    float* s_probe = reinterpret_cast<float*>(s_sum);      // [k][kKmProbes]: 256 bytes per centre, as the slots
    uint64_t* s_idx = reinterpret_cast<uint64_t*>(s_cnt);  // [k] seeded indices
    if (tid < k) s_idx[tid] = mix64(key + (uint64_t)(tid + 1) * kGolden) % un;
    __syncthreads();
    constexpr int PR = (KMAX * kKmProbes + NT - 1) / NT;  // probes per thread
    float probe[PR];
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        const int e = tid + r * NT;
        if (e < k * kKmProbes) {
            const int j = e / kKmProbes;
            const uint64_t t = s_idx[j] + (uint64_t)(e - j * kKmProbes);
            probe[r] = in[un > (uint64_t)kKmProbes ? (t >= un ? t - un : t) : t % un];
        }
    }
    float amax = 0.f;
    if (vec) {
        const float4* in4 = reinterpret_cast<const float4*>(in);
#pragma unroll 8
        for (long long i = tid; i < n / 4; i += NT) {
            const float4 a = __ldg(in4 + i);
            amax = fmaxf(amax, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
        }
    } else {
#pragma unroll 4
        for (long long i = tid; i < n; i += NT) amax = fmaxf(amax, fabsf(in[i]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(full, amax, o));
    if (lane == 0) reinterpret_cast<float*>(s_red)[warp] = amax;
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        const int e = tid + r * NT;
        if (e < k * kKmProbes) s_probe[e] = probe[r];
    }
    __syncthreads();
    if (warp == 0) {
        for (int j = 0; j < k; ++j) {
            float pick = s_probe[j * kKmProbes];
            for (int round = 0; round < kKmProbes / 32; ++round) {
                const float cand = s_probe[j * kKmProbes + round * 32 + lane];
                bool dup = false;
#pragma unroll
                for (int q = 0; q < KMAX; ++q) dup |= (q < j) && (s_cent[q] == cand);
                const unsigned bal = __ballot_sync(full, !dup);
                if (bal) {
                    pick = __shfl_sync(full, cand, __ffs(bal) - 1);
                    break;
                }
            }
            if (lane == 0) s_cent[j] = pick;
            __syncwarp();
        }
        // ascending order, equal values in index order (a stable sort): each centre's
        // rank among the k; NaN centres have no rank, so they take the insertion sort
        const float t = lane < k ? s_cent[lane] : 0.f;
        if (__any_sync(full, lane < k && isnan(t))) {
            if (lane == 0) {
                for (int j = 1; j < k; ++j) {
                    const float u = s_cent[j];
                    int q = j - 1;
                    while (q >= 0 && s_cent[q] > u) {
                        s_cent[q + 1] = s_cent[q];
                        --q;
                    }
                    s_cent[q + 1] = u;
                }
            }
        } else {
            int rank = 0;
#pragma unroll
            for (int q = 0; q < KMAX; ++q) {
                const float cq = s_cent[q];
                rank += (q < k && (cq < t || (cq == t && q < lane))) ? 1 : 0;
            }
            __syncwarp();
            if (lane < k) s_cent[rank] = t;
        }
        __syncwarp();
        if (lane >= k && lane < KMAX) s_cent[lane] = INFINITY;
        if (lane == 0) {
            s_cent[-2] = -INFINITY;
            s_cent[-1] = -INFINITY;
            s_cent[KMAX] = INFINITY;
        }
    }
    __syncthreads();
    for (int w = 0; w < NW; ++w) amax = fmaxf(amax, reinterpret_cast<const float*>(s_red)[w]);
    int lgn = 0;
    while (lgn < 62 && (1ll << lgn) < n) ++lgn;
    const int e = ((__float_as_int(amax) >> 23) & 0xff) - 126;  // amax < 2^e (e = -126 for amax = 0)
    const int sh = max(-126, min(127, 62 - lgn - e));
    const float scale = __int_as_float((sh + 127) << 23);
    __syncthreads();  // s_red, s_probe and s_idx are reused below

    for (int t = 0; t <= iters; ++t) {
        const bool last = (t == iters);
        if (!last)
            for (int e = tid; e < k * 32; e += NT) {
                if (split) {
#pragma unroll
                    for (int a = 0; a < 4; ++a) s_w32[a * CNT + e] = 0;
                } else {
                    s_sum[e] = 0;
                    s_cnt[e] = 0;
                }
            }
        __syncthreads();
        double J = 0.0;
        // One assignment pass over the input, four consecutive values per thread and
        // trip, the next trip's values loaded while this one's are assigned. The
        // switches are compile-time: the final pass (codes and deq) or a Lloyd pass
        // (member sums), 32-bit sum pieces with 32-bit indices, 16-byte access.
        auto pass = [&](auto zero, auto last_c, auto split_c, auto vec_c) {
            using I = decltype(zero);
            constexpr bool LAST = decltype(last_c)::value, SPLIT = decltype(split_c)::value;
            constexpr bool VEC = decltype(vec_c)::value;
            const I ni = (I)n;
            auto load4 = [&](float (&v)[4], I i0) {
                if (VEC) {
                    if (i0 < ni) {
                        const float4 a = __ldg(reinterpret_cast<const float4*>(in + i0));
                        v[0] = a.x;
                        v[1] = a.y;
                        v[2] = a.z;
                        v[3] = a.w;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] = i0 + q < ni ? in[i0 + q] : 0.f;
                }
            };
            float nv[4] = {0.f, 0.f, 0.f, 0.f};
            load4(nv, 4 * (I)tid);
            for (I i0 = 4 * (I)tid; i0 < ni; i0 += 4 * (I)NT) {
                float v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = nv[q];
                load4(nv, i0 + 4 * (I)NT);
                int best[4];
                bool walk[4];
                float dl[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) best[q] = nearest_centre_flat<KMAX>(s_cent, k, v[q], walk[q], dl[q]);
                if (walk[0] || walk[1] || walk[2] || walk[3]) {  // rare: duplicate or nearly equal centres
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (walk[q]) best[q] = walk_down(s_cent, best[q], v[q], dl[q]);
                }
                const int nq = VEC ? 4 : (int)min((I)4, ni - i0);  // values of this trip (4 but at a ragged tail)
                if (LAST) {
                    if (VEC) {
                        *reinterpret_cast<float4*>(deq + i0) =
                            make_float4(s_cent[best[0]], s_cent[best[1]], s_cent[best[2]], s_cent[best[3]]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (q < nq) deq[i0 + q] = s_cent[best[q]];
                    }
                    if (codes) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (q < nq) codes[i0 + q] = (uint8_t)best[q];
                    }
                } else {
                    // integer adds: exact, so the order in which the warps add does not matter
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int slot = 32 * (q < nq ? best[q] : KMAX) + lane;
                        const long long fx = __float2ll_rn(v[q] * scale);
                        if (SPLIT) {
                            const unsigned lo = (unsigned)fx;
                            atomicAdd(s_w32 + slot, (unsigned)(fx >> 32));
                            atomicAdd(s_w32 + CNT + slot, lo >> 16);
                            atomicAdd(s_w32 + 2 * CNT + slot, lo & 0xffffu);
                            atomicAdd(s_w32 + 3 * CNT + slot, 1u);
                        } else {
                            atomicAdd(s_sum + slot, (unsigned long long)fx);
                            atomicAdd(s_cnt + slot, 1ull);
                        }
                    }
                }
                if (obj) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (q < nq) {
                            const double d = (double)v[q] - (double)s_cent[best[q]];
                            J += d * d;
                        }
                }
            }
        };
        auto run = [&](auto last_c) {
            using T = std::true_type;
            using F = std::false_type;
            if (split) {  // n < 2^21: 32-bit indices as well
                if (vec) pass(0, last_c, T{}, T{});
                else pass(0, last_c, T{}, F{});
            } else {
                if (vec) pass(0ll, last_c, F{}, T{});
                else pass(0ll, last_c, F{}, F{});
            }
        };
        if (last) run(std::true_type{});
        else run(std::false_type{});
        if (obj) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) J += __shfl_xor_sync(full, J, o);
            if (lane == 0) s_red[warp] = J;
            __syncthreads();
            if (tid == 0) {
                double tot = 0.0;
                for (int w = 0; w < NW; ++w) tot += s_red[w];
                obj[t] = tot;
            }
        }
        if (last) break;
        __syncthreads();
        // centre update: the exact member sum over the lanes' slots, mean in FP64; eight
        // threads per centre (each adds four lanes' slots), so that every centre's
        // division runs at once
        static_assert(8 * KMAX <= NT, "eight threads per centre");
        if (tid < 8 * KMAX) {
            const int j = tid >> 3, g = tid & 7;
            long long sm = 0;
            int c = 0;
            if (j < k) {
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const int e = j * 32 + 4 * g + l;
                    if (split) {
                        sm += (long long)(int)s_w32[e] * 4294967296ll + (long long)s_w32[CNT + e] * 65536ll +
                              (long long)s_w32[2 * CNT + e];
                        c += (int)s_w32[3 * CNT + e];
                    } else {
                        sm += (long long)s_sum[e];
                        c += (int)s_cnt[e];
                    }
                }
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                sm += __shfl_xor_sync(full, sm, o);
                c += __shfl_xor_sync(full, c, o);
            }
            if (g == 0 && j < k && c > 0) s_cent[j] = (float)ldexp((double)sm / (double)c, -sh);
        }
        __syncthreads();
    }
    if (cent_out && tid < k) cent_out[tid] = s_cent[tid];
}

template <int KMAX>
__global__ void __launch_bounds__(kKmThreads, 4) kmeans_single_kernel(const float* in, long long n, int k,
                                                                   int iters, uint64_t key, uint8_t* codes,
                                                                   float* cent, float* deq, double* obj) {
    kmeans_block<KMAX>(in, n, k, iters, key, codes, cent, deq, obj);
}

template <int KMAX>
__global__ void __launch_bounds__(kKmThreads, 4) kmeans_dadmm_kernel(const DadmmCodec p, int k, int iters,
                                                                  int task_begin) {
    const SegTask T = p.tasks[task_begin + blockIdx.x];
    const int kk = *p.iter;  // completed iterations: the messages are x^{k+1}
    const long long len = (long long)(T.r1 - T.r0) * p.N;
    const int slot = (kk + 1) % p.D;
    float* deq = p.hist + (size_t)slot * p.slot_stride + (size_t)DADMM_Q_KMEANS * p.plane_stride + T.dst_off;
    kmeans_block<KMAX>(p.xseg + T.src_off, len, k, iters, kmeans_key(p.seed, T.slice, T.owner, kk + 1),
                       nullptr, nullptr, deq, nullptr);
}

template <class F>
static void with_kmax(int k, F&& f) {
    if (k <= 8)
        f(std::integral_constant<int, 8>());
    else if (k <= 16)
        f(std::integral_constant<int, 16>());
    else
        f(std::integral_constant<int, 32>());
}

// dynamic shared-memory opt-in of the K-means kernels, once per process and
// template instance, always before any stream capture
template <int KMAX>
static void ensure_km_attr() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        const int sm = (int)kmeans_smem(KMAX);
        err = cudaFuncSetAttribute(kmeans_single_kernel<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(kmeans_dadmm_kernel<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    });
    TOMO_CUDA(err);
}

void launch_kmeans_single(const float* in, long long n, int k, int iters, uint64_t key, uint8_t* codes,
                          float* cent, float* deq, double* obj, cudaStream_t st) {
    with_kmax(k, [&](auto KM) {
        constexpr int KMAX = decltype(KM)::value;
        const size_t sm = kmeans_smem(KMAX);
        ensure_km_attr<KMAX>();
        kmeans_single_kernel<KMAX><<<1, kKmThreads, sm, st>>>(in, n, k, iters, key, codes, cent, deq, obj);
        TOMO_CUDA(cudaGetLastError());
    });
}

void launch_kmeans_dadmm(const DadmmCodec& p, int k, int iters, int task_begin, int task_count,
                         cudaStream_t st) {
    if (task_count <= 0) return;
    with_kmax(k, [&](auto KM) {
        constexpr int KMAX = decltype(KM)::value;
        const size_t sm = kmeans_smem(KMAX);
        ensure_km_attr<KMAX>();
        kmeans_dadmm_kernel<KMAX><<<task_count, kKmThreads, sm, st>>>(p, k, iters, task_begin);
        TOMO_CUDA(cudaGetLastError());
    });
}

// ------------------------------------------------------------------
// JPEG
// ------------------------------------------------------------------

// ITU-T T.81 (1992) Annex K, Table K.1, luminance, natural order
static const int kJpegLuma[64] = {16, 11, 10, 16, 24,  40,  51,  61,  12, 12, 14, 19, 26,  58,  60,  55,
                                  14, 13, 16, 24, 40,  57,  69,  56,  14, 17, 22, 29, 51,  87,  80,  62,
                                  18, 22, 37, 56, 68,  109, 103, 77,  24, 35, 55, 64, 81,  104, 113, 92,
                                  49, 64, 78, 87, 103, 121, 120, 101, 72, 92, 95, 98, 112, 100, 103, 99};

void jpeg_quant_table(int quality, int32_t* qt) {
    quality = quality < 1 ? 1 : quality > 100 ? 100 : quality;
    const int scale = quality < 50 ? 5000 / quality : 200 - 2 * quality;  // IJG rule
    for (int i = 0; i < 64; ++i) {
        const long v = ((long)kJpegLuma[i] * scale + 50) / 100;
        qt[i] = (int32_t)(v < 1 ? 1 : v > 255 ? 255 : v);
    }
}

// basis[p][x] = C(p)/2 cos((2x+1) p pi / 16), C(0) = 1/sqrt(2); FP32 for
// the transforms, FP64 for re-deciding the rare near-tie roundings
__constant__ float c_dct[64];
__constant__ double c_dct64[64];

static void ensure_dct_table() {
    static std::mutex mu;
    static std::vector<char> done;
    int dev = 0;
    TOMO_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)done.size() <= dev) done.resize(dev + 1, 0);
    if (done[dev]) return;
    float h[64];
    double h64[64];
    for (int p = 0; p < 8; ++p)
        for (int x = 0; x < 8; ++x) {
            h64[p * 8 + x] = (p == 0 ? 1.0 / std::sqrt(2.0) : 1.0) * 0.5 *
                             std::cos((2 * x + 1) * p * 3.14159265358979323846 / 16.0);
            h[p * 8 + x] = (float)h64[p * 8 + x];
        }
    TOMO_CUDA(cudaMemcpyToSymbol(c_dct, h, sizeof(h)));
    TOMO_CUDA(cudaMemcpyToSymbol(c_dct64, h64, sizeof(h64)));
    done[dev] = 1;
}

struct QTable {
    int q[64];
};

constexpr int kJpegThreads = 64;

// Bound of the FP32 error of one output of the separable 8x8 transform of
// inputs x (|basis| <= 1/2, 8 + 8 accumulated FMAs with rounded basis values):
// 2 gamma_9 (1/2)^2 sum|x| ~ 2.7e-7 sum|x|; taken 4x larger. A rounding
// decision whose FP32 value lies closer than that to the tie is re-decided
// in FP64.
__device__ __forceinline__ float fp32_transform_bound(float sum_abs) { return 1.1e-6f * sum_abs + 1e-6f; }

// sign of cos((2i+1) pi / 4): the basis of frequency 4 up to 1/(2 sqrt 2)
__device__ constexpr float kSigma4[8] = {1.f, -1.f, -1.f, 1.f, 1.f, -1.f, -1.f, 1.f};

// coefficients (p, q) with p, q in {0, 4}: weights +-1/8, rational values
__device__ __forceinline__ bool is_rational(int e) { return e == 0 || e == 4 || e == 32 || e == 36; }

// distance of x to the nearest half-integer multiple of q: |x| - (k + 1/2) q
__device__ __forceinline__ float tie_distance(float x, float q) {
    const float ax = fabsf(x);
    const float k = floorf(ax / q);
    return fabsf(ax - (k + 0.5f) * q);
}

// one 8x8 block: src/dst point at its top-left value, `stride` floats per row;
// s_smp / s_q: this thread's 64-entry scratch in shared memory, element e at
// [e * kJpegThreads] (transposed: conflict-free across the warp).
// Returns the number of non-zero quantized coefficients.
__device__ __forceinline__ int jpeg_block(const float* __restrict__ src, float* __restrict__ dst, int stride,
                                          float lo, float hi, const QTable& qt, int16_t* coefs,
                                          int8_t* s_smp, int16_t* s_q) {
    const float rng = __fsub_rn(hi, lo);
    const float inv = __fdiv_rn(255.0f, rng);
    const float step = __fdiv_rn(rng, 255.0f);
    float b[64];
    // integer sums of the samples (exact in FP32): the coefficients (0,0),
    // (0,4), (4,0), (4,4) have weights +-1/8 and are formed exactly from them
    float f00 = 0.f, f04 = 0.f, f40 = 0.f, f44 = 0.f, sabs = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 v0 = *reinterpret_cast<const float4*>(src + (size_t)i * stride);
        const float4 v1 = *reinterpret_cast<const float4*>(src + (size_t)i * stride + 4);
        const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        float rs = 0.f, r4 = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float t = __fmul_rn(__fsub_rn(v[j], lo), inv);
            const float r = fminf(fmaxf(roundf(t), 0.0f), 255.0f);  // round half away from zero
            b[i * 8 + j] = r - 128.0f;
            s_smp[(i * 8 + j) * kJpegThreads] = (int8_t)(int)(r - 128.0f);
            rs += b[i * 8 + j];
            r4 += kSigma4[j] * b[i * 8 + j];
            sabs += fabsf(b[i * 8 + j]);
        }
        f00 += rs;
        f40 += kSigma4[i] * rs;
        f04 += r4;
        f44 += kSigma4[i] * r4;
    }
    // forward DCT: rows, then columns
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float t[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) t[j] = b[i * 8 + j];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float a = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) a = fmaf(t[j], c_dct[q * 8 + j], a);
            b[i * 8 + q] = a;
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float t[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = b[i * 8 + q];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) a = fmaf(c_dct[p * 8 + i], t[i], a);
            b[p * 8 + q] = a;
        }
    }
    b[0] = f00 * 0.125f;  // exact: ties of F / Qt are decided by the rounding rule
    b[4] = f04 * 0.125f;
    b[32] = f40 * 0.125f;
    b[36] = f44 * 0.125f;
    const float dF = fp32_transform_bound(sabs);
    unsigned long long near = 0ull;
#pragma unroll
    for (int e = 0; e < 64; ++e) {
        const float Q = (float)qt.q[e];
        const float qv = roundf(__fdiv_rn(b[e], Q));
        if (!is_rational(e) && tie_distance(b[e], Q) < dF) near |= 1ull << e;
        s_q[e * kJpegThreads] = (int16_t)fminf(fmaxf(qv, -32768.0f), 32767.0f);
    }
    while (near) {  // re-decide near-tie coefficients from the samples in FP64
        const int e = __ffsll((long long)near) - 1;
        near &= near - 1;
        const int p = e >> 3, q = e & 7;
        double F = 0.0;
        for (int i = 0; i < 8; ++i) {
            double r = 0.0;
            for (int j = 0; j < 8; ++j) r = fma((double)s_smp[(i * 8 + j) * kJpegThreads], c_dct64[q * 8 + j], r);
            F = fma(c_dct64[p * 8 + i], r, F);
        }
        s_q[e * kJpegThreads] = (int16_t)fmin(fmax(round(F / (double)qt.q[e]), -32768.0), 32767.0);
    }
    int nnz = 0;
    float gabs = 0.f;
#pragma unroll
    for (int e = 0; e < 64; ++e) {
        const int qv = s_q[e * kJpegThreads];
        if (coefs) coefs[e] = (int16_t)qv;
        nnz += (qv != 0);
        b[e] = (float)(qv * qt.q[e]);  // integer product: exact
        if (!is_rational(e)) gabs += fabsf(b[e]);
    }
    // the rational part of every output value, exact: (G00 + s4(j) G04 + s4(i) G40 + s4(i) s4(j) G44) / 8
    const float g00 = b[0], g04 = b[4], g40 = b[32], g44 = b[36];
    b[0] = b[4] = b[32] = b[36] = 0.f;
    const float dS = fp32_transform_bound(gabs);
    // inverse DCT of the AC part: columns, then rows
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float t[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) t[p] = b[p * 8 + q];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float a = 0.f;
#pragma unroll
            for (int p = 0; p < 8; ++p) a = fmaf(c_dct[p * 8 + i], t[p], a);
            b[i * 8 + q] = a;
        }
    }
    near = 0ull;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float t[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) t[q] = b[i * 8 + q];
        float o[8];
        const float ra = g00 + kSigma4[i] * g40, rb = g04 + kSigma4[i] * g44;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float a = 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q) a = fmaf(t[q], c_dct[q * 8 + j], a);
            const float rat = (ra + kSigma4[j] * rb) * 0.125f + 128.0f;  // exact
            const float v = a + rat;
            if (fabsf(v - floorf(v) - 0.5f) < dS) near |= 1ull << (i * 8 + j);
            const float r = fminf(fmaxf(roundf(v), 0.0f), 255.0f);
            o[j] = (r == 255.0f) ? hi : __fadd_rn(lo, __fmul_rn(r, step));
        }
        *reinterpret_cast<float4*>(dst + (size_t)i * stride) = make_float4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<float4*>(dst + (size_t)i * stride + 4) = make_float4(o[4], o[5], o[6], o[7]);
    }
    while (near) {  // re-decide near-tie samples from the quantized coefficients in FP64
        const int e = __ffsll((long long)near) - 1;
        near &= near - 1;
        const int i = e >> 3, j = e & 7;
        double v = 0.0;
        for (int p = 0; p < 8; ++p) {
            double r = 0.0;
            for (int q = 0; q < 8; ++q)
                if (!is_rational(p * 8 + q))
                    r = fma((double)(s_q[(p * 8 + q) * kJpegThreads] * qt.q[p * 8 + q]), c_dct64[q * 8 + j], r);
            v = fma(c_dct64[p * 8 + i], r, v);
        }
        v += ((double)g00 + kSigma4[i] * (double)g40 + kSigma4[j] * ((double)g04 + kSigma4[i] * (double)g44)) * 0.125 +
             128.0;
        const float r = (float)fmin(fmax(round(v), 0.0), 255.0);
        dst[(size_t)i * stride + j] = (r == 255.0f) ? hi : __fadd_rn(lo, __fmul_rn(r, step));
    }
    return nnz;
}

__device__ __forceinline__ void jpeg_const_block(float* dst, int stride, float lo) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        *reinterpret_cast<float4*>(dst + (size_t)i * stride) = make_float4(lo, lo, lo, lo);
        *reinterpret_cast<float4*>(dst + (size_t)i * stride + 4) = make_float4(lo, lo, lo, lo);
    }
}

// min / max of one segment with one block (standalone path)
__global__ void minmax_kernel(const float* in, long long n, float* lohi) {
    __shared__ float s_lo[32], s_hi[32];
    float lo = INFINITY, hi = -INFINITY;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        lo = fminf(lo, in[i]);
        hi = fmaxf(hi, in[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = fminf(lo, s_lo[w]);
            hi = fmaxf(hi, s_hi[w]);
        }
        lohi[0] = lo;
        lohi[1] = hi;
    }
}

__global__ void __launch_bounds__(kJpegThreads) jpeg_single_kernel(const float* in, int rows, int cols,
                                                                   const QTable qt, int16_t* coefs,
                                                                   const float* lohi, float* deq,
                                                                   long long* nnz) {
    __shared__ int8_t s_smp[64][kJpegThreads];
    __shared__ int16_t s_q[64][kJpegThreads];
    const int bpr = cols / 8;
    const int blk = blockIdx.x * kJpegThreads + threadIdx.x;
    int c = 0;
    if (blk < (rows / 8) * bpr) {
        const int bi = blk / bpr, bj = blk - bi * bpr;
        const size_t o = (size_t)bi * 8 * cols + (size_t)bj * 8;
        const float lo = lohi[0], hi = lohi[1];
        int16_t* cf = coefs ? coefs + (size_t)blk * 64 : nullptr;
        if (hi > lo) {
            c = jpeg_block(in + o, deq + o, cols, lo, hi, qt, cf, &s_smp[0][threadIdx.x], &s_q[0][threadIdx.x]);
        } else {
            jpeg_const_block(deq + o, cols, lo);
            if (cf)
                for (int e = 0; e < 64; ++e) cf[e] = 0;
        }
    }
    if (nnz) {
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long*)nnz, (unsigned long long)c);
    }
}

__global__ void __launch_bounds__(kJpegThreads) jpeg_dadmm_kernel(const DadmmCodec p, const QTable qt,
                                                                  int task_begin) {
    __shared__ int8_t s_smp[64][kJpegThreads];
    __shared__ int16_t s_q[64][kJpegThreads];
    const SegTask T = p.tasks[task_begin + blockIdx.y];
    const int N = p.N, bpr = N / 8;
    const int blk = blockIdx.x * kJpegThreads + threadIdx.x;
    if (blk < ((T.r1 - T.r0) / 8) * bpr) {
        const int kk = *p.iter;
        const int bi = blk / bpr, bj = blk - bi * bpr;
        const size_t o = (size_t)(bi * 8) * N + (size_t)bj * 8;  // within the segment
        const int slot = (kk + 1) % p.D;
        float* dst = p.hist + (size_t)slot * p.slot_stride + (size_t)DADMM_Q_JPEG * p.plane_stride + T.dst_off + o;
        const float lo = key_float(p.lo_key[T.slice * p.M + T.owner]);
        const float hi = key_float(p.hi_key[T.slice * p.M + T.owner]);
        int16_t* cf = p.coefs + ((size_t)T.blk0 + blk) * 64;
        if (hi > lo) {
            jpeg_block(p.xseg + T.src_off + o, dst, N, lo, hi, qt, cf, &s_smp[0][threadIdx.x], &s_q[0][threadIdx.x]);
        } else {
            jpeg_const_block(dst, N, lo);
            for (int e = 0; e < 64; ++e) cf[e] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Baseline Huffman entropy coding of quantized 8x8 blocks (ITU-T T.81 Annex
// F.1.2: DC difference categories + extra bits, AC run/size symbols with ZRL
// and EOB in zig-zag order) with the luminance tables of Annex K (K.3 DC,
// K.5 AC), codes assigned canonically (Annex C). One CTA per image: the
// blocks' bit lengths are scanned across the CTA 256 blocks at a time, every
// thread packs its block's codes at its bit offset into a zeroed word
// buffer (stream bit 0 = the MSB of word 0; atomicOr where two blocks share
// a word), the last byte is padded with 1-bits, and every 0xFF byte is
// followed by a stuffed 0x00 (counted; written when a stream is requested).
// ---------------------------------------------------------------------------
namespace {
const uint8_t kDcBits[16] = {0, 1, 5, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0};
const uint8_t kAcBits[16] = {0, 2, 1, 3, 3, 2, 4, 3, 5, 5, 4, 4, 0, 0, 1, 125};
const uint8_t kAcVals[162] = {
    0x01, 0x02, 0x03, 0x00, 0x04, 0x11, 0x05, 0x12, 0x21, 0x31, 0x41, 0x06, 0x13, 0x51, 0x61, 0x07, 0x22, 0x71,
    0x14, 0x32, 0x81, 0x91, 0xa1, 0x08, 0x23, 0x42, 0xb1, 0xc1, 0x15, 0x52, 0xd1, 0xf0, 0x24, 0x33, 0x62, 0x72,
    0x82, 0x09, 0x0a, 0x16, 0x17, 0x18, 0x19, 0x1a, 0x25, 0x26, 0x27, 0x28, 0x29, 0x2a, 0x34, 0x35, 0x36, 0x37,
    0x38, 0x39, 0x3a, 0x43, 0x44, 0x45, 0x46, 0x47, 0x48, 0x49, 0x4a, 0x53, 0x54, 0x55, 0x56, 0x57, 0x58, 0x59,
    0x5a, 0x63, 0x64, 0x65, 0x66, 0x67, 0x68, 0x69, 0x6a, 0x73, 0x74, 0x75, 0x76, 0x77, 0x78, 0x79, 0x7a, 0x83,
    0x84, 0x85, 0x86, 0x87, 0x88, 0x89, 0x8a, 0x92, 0x93, 0x94, 0x95, 0x96, 0x97, 0x98, 0x99, 0x9a, 0xa2, 0xa3,
    0xa4, 0xa5, 0xa6, 0xa7, 0xa8, 0xa9, 0xaa, 0xb2, 0xb3, 0xb4, 0xb5, 0xb6, 0xb7, 0xb8, 0xb9, 0xba, 0xc2, 0xc3,
    0xc4, 0xc5, 0xc6, 0xc7, 0xc8, 0xc9, 0xca, 0xd2, 0xd3, 0xd4, 0xd5, 0xd6, 0xd7, 0xd8, 0xd9, 0xda, 0xe1, 0xe2,
    0xe3, 0xe4, 0xe5, 0xe6, 0xe7, 0xe8, 0xe9, 0xea, 0xf1, 0xf2, 0xf3, 0xf4, 0xf5, 0xf6, 0xf7, 0xf8, 0xf9, 0xfa};
// zig-zag position -> natural index (row * 8 + column)
const uint8_t kZigzag[64] = {0,  1,  8,  16, 9,  2,  3,  10, 17, 24, 32, 25, 18, 11, 4,  5,
                             12, 19, 26, 33, 40, 48, 41, 34, 27, 20, 13, 6,  7,  14, 21, 28,
                             35, 42, 49, 56, 57, 50, 43, 36, 29, 22, 15, 23, 30, 37, 44, 51,
                             58, 59, 52, 45, 38, 31, 39, 46, 53, 60, 61, 54, 47, 55, 62, 63};
}  // namespace

struct HuffTables {
    uint32_t dc[12];   // (code << 8) | length of each DC category
    uint32_t ac[256];  // (code << 8) | length of each run/size symbol (length 0: none)
    uint8_t zz[64];
};

static const HuffTables& huff_tables() {
    static HuffTables t;
    static std::once_flag once;
    std::call_once(once, [] {
        std::memset(&t, 0, sizeof(t));
        auto build = [](const uint8_t* bits, const uint8_t* vals, uint32_t* out) {
            uint32_t code = 0;
            int k = 0;
            for (int l = 1; l <= 16; ++l) {
                for (int i = 0; i < bits[l - 1]; ++i, ++k) out[vals ? vals[k] : k] = (code++ << 8) | (uint32_t)l;
                code <<= 1;
            }
        };
        build(kDcBits, nullptr, t.dc);
        build(kAcBits, kAcVals, t.ac);
        std::memcpy(t.zz, kZigzag, 64);
    });
    return t;
}

struct EntropyTask {
    long long blk0;   // first block in the coefficient buffer
    long long word0;  // first word of the bit buffer (kEntropyWordsPerBlock per block)
    int nblk;
    int out;          // index of the byte count to write
    int lohi;         // >= 0: index of the (lo, hi) keys; a constant segment codes to 0 bytes
    int pad;
};

struct EntropyParams {
    HuffTables t;
    const int16_t* coefs;
    EntropyTask one;      // the task when seg is null (standalone call: one CTA)
    const SegTask* seg;   // dADMM: one CTA per JPEG segment
    uint32_t* bits;
    long long* bytes;     // out: stream length in bytes (stuffed), -1 if a coefficient is out of range
    const unsigned* lo_key;
    const unsigned* hi_key;
    uint8_t* stream;      // optional: the stuffed stream (single task)
    int N, M;             // dADMM: image width, nodes
};

__device__ __forceinline__ uint32_t extra_bits(int v, int s) {
    return (uint32_t)(v >= 0 ? v : v - 1) & ((1u << s) - 1u);
}

__device__ __forceinline__ int category(int v) { return 32 - __clz(v < 0 ? -v : v); }

// codes of one block as (value, length) pairs, value = code word then extra bits;
// returns false if a coefficient is outside the baseline range
template <class Emit>
__device__ __forceinline__ bool code_block(const int16_t* c, int pred, const uint32_t* dc, const uint32_t* ac,
                                           const uint8_t* zz, Emit emit) {
    const int diff = c[0] - pred;
    const int sd = category(diff);
    if (sd > 11) return false;
    emit(((dc[sd] >> 8) << sd) | extra_bits(diff, sd), (int)(dc[sd] & 255u) + sd);
    int run = 0;
    for (int k = 1; k < 64; ++k) {
        const int v = c[zz[k]];
        if (v == 0) {
            ++run;
            continue;
        }
        for (; run > 15; run -= 16) emit(ac[0xF0] >> 8, (int)(ac[0xF0] & 255u));
        const int sa = category(v);
        if (sa > 10) return false;
        const uint32_t a = ac[(run << 4) | sa];
        emit(((a >> 8) << sa) | extra_bits(v, sa), (int)(a & 255u) + sa);
        run = 0;
    }
    if (run) emit(ac[0] >> 8, (int)(ac[0] & 255u));  // EOB
    return true;
}

// stream bits [o, o + len) = the low len bits of v, MSB first (len <= 27)
__device__ __forceinline__ void put_bits(uint32_t* buf, unsigned long long o, uint32_t v, int len) {
    const unsigned long long x = (unsigned long long)v << (64 - (int)(o & 31) - len);
    atomicOr(buf + (o >> 5), (uint32_t)(x >> 32));
    if ((uint32_t)x) atomicOr(buf + (o >> 5) + 1, (uint32_t)x);
}

// threads of the entropy coder's CTA: each codes a contiguous run of 8 x 8 blocks
// (4 of a 1024-block segment)
constexpr int kEntThreads = 256;

// CTA-wide exclusive scan of one value per thread (kEntThreads threads); returns the
// prefix and sets *total
__device__ __forceinline__ long long cta_exclusive_scan(long long v, long long* total) {
    __shared__ long long s_w[kEntThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    long long before = 0, all = 0;
    for (int w = 0; w < kEntThreads / 32; ++w) {
        if (w < warp) before += s_w[w];
        all += s_w[w];
    }
    __syncthreads();  // s_w reused by the next call
    *total = all;
    return before + x - v;
}

__global__ void __launch_bounds__(kEntThreads) jpeg_entropy_kernel(const __grid_constant__ EntropyParams p) {
    __shared__ uint32_t s_dc[12], s_ac[256];
    __shared__ uint8_t s_zz[64];
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    for (int i = tid; i < 256; i += kEntThreads) s_ac[i] = p.t.ac[i];
    if (tid < 12) s_dc[tid] = p.t.dc[tid];
    if (tid < 64) s_zz[tid] = p.t.zz[tid];
    if (tid == 0) s_bad = 0;
    EntropyTask T;
    if (p.seg) {
        const SegTask S = p.seg[blockIdx.x];
        T.blk0 = S.blk0;
        T.word0 = S.word0;
        T.nblk = ((S.r1 - S.r0) / 8) * (p.N / 8);
        T.out = S.slice * p.M + S.owner;
        T.lohi = T.out;
    } else {
        T = p.one;
    }
    __syncthreads();
    if (T.lohi >= 0 && !(key_float(p.hi_key[T.lohi]) > key_float(p.lo_key[T.lohi]))) {
        if (tid == 0) p.bytes[T.out] = 0;  // a constant segment is sent as its value alone
        return;
    }
    // Each thread codes a contiguous run of blocks twice: once to size it, and,
    // after one scan of the runs' sizes has given every run its bit offset, once to
    // write it. Only the words the stream occupies are cleared (the rest of the
    // buffer is never read).
    uint32_t* buf = p.bits + T.word0;
    const long long nwords = (long long)T.nblk * kEntropyWordsPerBlock + 1;
    const int16_t* coefs = p.coefs + T.blk0 * 64;
    const int per = (T.nblk + kEntThreads - 1) / kEntThreads;
    const int bb = min(T.nblk, tid * per), be = min(T.nblk, bb + per);
    long long nbits = 0;
    for (int b = bb; b < be; ++b) {
        const int pred = b > 0 ? coefs[(size_t)(b - 1) * 64] : 0;
        int nb = 0;
        if (!code_block(coefs + (size_t)b * 64, pred, s_dc, s_ac, s_zz, [&](uint32_t, int len) { nb += len; }))
            atomicOr(&s_bad, 1);
        nbits += nb;
    }
    long long total;
    const long long at = cta_exclusive_scan(nbits, &total);
    const long long used = min((total >> 5) + 2, nwords);  // the stream and its padding
    for (long long i = tid; i < used; i += kEntThreads) buf[i] = 0u;
    __syncthreads();
    unsigned long long o = (unsigned long long)at;
    for (int b = bb; b < be; ++b) {
        const int pred = b > 0 ? coefs[(size_t)(b - 1) * 64] : 0;
        code_block(coefs + (size_t)b * 64, pred, s_dc, s_ac, s_zz, [&](uint32_t v, int len) {
            if (len > 0) put_bits(buf, o, v, len);
            o += len;
        });
    }
    const unsigned long long base = (unsigned long long)total;
    if (tid == 0 && (base & 7)) {  // pad the last byte with 1-bits
        const int pad = 8 - (int)(base & 7);
        put_bits(buf, base, (1u << pad) - 1u, pad);
    }
    __threadfence();
    __syncthreads();
    if (s_bad) {
        if (tid == 0) p.bytes[T.out] = -1;
        return;
    }
    // 0xFF bytes of the stream, each followed by a stuffed zero
    const unsigned long long nbytes = (base + 7) >> 3;
    const long long nw = (long long)((nbytes + 3) >> 2);
    unsigned long long out_pos = 0;
    if (!p.stream) {  // the byte count only: one reduction over the words
        long long cnt = 0;
        for (long long w = tid; w < nw; w += kEntThreads) {
            const uint32_t word = __ldcg(buf + w);
            const int nb = (int)min(4ull, nbytes - 4ull * (unsigned long long)w);
            cnt += nb;
            for (int q = 0; q < nb; ++q) cnt += ((word >> (24 - 8 * q)) & 255u) == 255u;
        }
        long long all;
        cta_exclusive_scan(cnt, &all);
        if (tid == 0) p.bytes[T.out] = all;
        return;
    }
    for (long long w0 = 0; w0 < nw; w0 += kEntThreads) {
        const long long w = w0 + tid;
        uint32_t word = 0;
        int nb = 0, ff = 0;
        if (w < nw) {
            word = __ldcg(buf + w);
            nb = (int)min(4ull, nbytes - 4ull * (unsigned long long)w);
            for (int q = 0; q < nb; ++q) ff += ((word >> (24 - 8 * q)) & 255u) == 255u;
        }
        long long total;
        const long long before = cta_exclusive_scan(nb + ff, &total);
        if (p.stream && w < nw) {
            unsigned long long o = out_pos + before;
            for (int q = 0; q < nb; ++q) {
                const uint8_t byte = (uint8_t)(word >> (24 - 8 * q));
                p.stream[o++] = byte;
                if (byte == 255u) p.stream[o++] = 0;
            }
        }
        out_pos += (unsigned long long)total;
    }
    if (tid == 0) p.bytes[T.out] = (long long)out_pos;
}

void launch_jpeg_entropy_dadmm(const DadmmCodec& c, int task_begin, int task_count, cudaStream_t st) {
    if (task_count <= 0) return;
    EntropyParams p{};
    p.t = huff_tables();
    p.coefs = c.coefs;
    p.seg = c.tasks + task_begin;
    p.bits = c.bits;
    p.bytes = c.jbytes;
    p.lo_key = c.lo_key;
    p.hi_key = c.hi_key;
    p.N = c.N;
    p.M = c.M;
    jpeg_entropy_kernel<<<task_count, kEntThreads, 0, st>>>(p);
    TOMO_CUDA(cudaGetLastError());
}

static float* lohi_scratch() {
    static std::mutex mu;
    static std::vector<float*> bufs;
    int dev = 0;
    TOMO_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)bufs.size() <= dev) bufs.resize(dev + 1, nullptr);
    if (!bufs[dev]) TOMO_CUDA(cudaMalloc(&bufs[dev], 256));  // once per device, held until exit
    return bufs[dev];
}

void launch_jpeg_single(const float* in, int rows, int cols, int quality, int16_t* coefs, float* lohi,
                        float* deq, long long* nnz, cudaStream_t st) {
    ensure_dct_table();
    float* lh = lohi ? lohi : lohi_scratch();
    minmax_kernel<<<1, 1024, 0, st>>>(in, (long long)rows * cols, lh);
    TOMO_CUDA(cudaGetLastError());
    QTable qt;
    jpeg_quant_table(quality, qt.q);
    const int nblk = (rows / 8) * (cols / 8);
    jpeg_single_kernel<<<ceil_div(nblk, kJpegThreads), kJpegThreads, 0, st>>>(in, rows, cols, qt, coefs, lh,
                                                                              deq, nnz);
    TOMO_CUDA(cudaGetLastError());
}

void launch_jpeg_dadmm(const DadmmCodec& p, int quality, int max_rows, int task_begin, int task_count,
                       cudaStream_t st) {
    if (task_count <= 0) return;
    ensure_dct_table();
    QTable qt;
    jpeg_quant_table(quality, qt.q);
    const int nblk = (max_rows / 8) * (p.N / 8);
    dim3 grid(ceil_div(nblk, kJpegThreads), task_count);
    jpeg_dadmm_kernel<<<grid, kJpegThreads, 0, st>>>(p, qt, task_begin);
    TOMO_CUDA(cudaGetLastError());
}

// everything that must not run while a stream is being captured
void prepare_codecs(int km_k) {
    ensure_dct_table();
    with_kmax(km_k < 1 ? 1 : km_k, [&](auto KM) { ensure_km_attr<decltype(KM)::value>(); });
}

}  // namespace tomo

using namespace tomo;

extern "C" {

uint64_t quant_kmeans_key(uint64_t seed, int slice, int owner, int iteration) {
    return tomo::kmeans_key(seed, slice, owner, iteration);
}

tomo_status quant_kmeans(const float* in, int64_t n, int k, int iters, uint64_t key, uint8_t* codes,
                         float* centroids, float* deq, double* objective, tomo_stream_t stream) {
    return guard([&] {
        TOMO_REQUIRE(in && deq, "in and deq must be non-NULL");
        TOMO_REQUIRE(n >= 1 && n <= (int64_t)1 << 40, "n out of range");
        TOMO_REQUIRE(k >= 1 && k <= kKmMaxK, "k must be in [1, 32]");
        TOMO_REQUIRE(iters >= 0 && iters <= 10000, "iters out of range");
        launch_kmeans_single(in, n, k, iters, key, codes, centroids, deq, objective, (cudaStream_t)stream);
    });
}

size_t quant_jpeg_entropy_bound(int rows, int cols) {
    if (rows < 8 || cols < 8) return 0;
    const size_t nblk = (size_t)(rows / 8) * (cols / 8);
    return 2 * (nblk * kEntropyWordsPerBlock * 4 + 4);  // every byte stuffed, at worst
}

size_t quant_jpeg_entropy_workspace_size(int rows, int cols) {
    if (rows < 8 || cols < 8) return 0;
    const size_t nblk = (size_t)(rows / 8) * (cols / 8);
    return (nblk * kEntropyWordsPerBlock + 1) * sizeof(uint32_t);
}

tomo_status quant_jpeg_entropy(const int16_t* coefs, int rows, int cols, uint8_t* stream, size_t stream_cap,
                               int64_t* nbytes, void* workspace, size_t workspace_bytes, tomo_stream_t st) {
    return guard([&] {
        TOMO_REQUIRE(coefs && nbytes, "coefs and nbytes must be non-NULL");
        TOMO_REQUIRE(rows >= 8 && cols >= 8 && rows % 8 == 0 && cols % 8 == 0,
                     "rows and cols must be positive multiples of 8");
        TOMO_REQUIRE(workspace && workspace_bytes >= quant_jpeg_entropy_workspace_size(rows, cols),
                     "workspace too small");
        TOMO_REQUIRE(((uintptr_t)workspace % 4) == 0, "workspace must be 4-byte aligned");
        TOMO_REQUIRE(!stream || stream_cap >= quant_jpeg_entropy_bound(rows, cols),
                     "stream capacity below quant_jpeg_entropy_bound()");
        EntropyParams p{};
        p.t = huff_tables();
        p.coefs = coefs;
        p.one.blk0 = 0;
        p.one.word0 = 0;
        p.one.nblk = (rows / 8) * (cols / 8);
        p.one.out = 0;
        p.one.lohi = -1;
        p.bits = (uint32_t*)workspace;
        p.bytes = (long long*)nbytes;
        p.stream = stream;
        jpeg_entropy_kernel<<<1, kEntThreads, 0, (cudaStream_t)st>>>(p);
        TOMO_CUDA(cudaGetLastError());
    });
}

tomo_status quant_jpeg(const float* in, int rows, int cols, int quality, int16_t* coefs, float* lohi,
                       float* deq, int64_t* nnz, tomo_stream_t stream) {
    return guard([&] {
        TOMO_REQUIRE(in && deq, "in and deq must be non-NULL");
        TOMO_REQUIRE(rows >= 8 && cols >= 8 && rows % 8 == 0 && cols % 8 == 0,
                     "rows and cols must be positive multiples of 8");
        TOMO_REQUIRE(quality >= 1 && quality <= 100, "quality must be in [1, 100]");
        TOMO_REQUIRE(((uintptr_t)in % 16) == 0 && ((uintptr_t)deq % 16) == 0,
                     "in and deq must be 16-byte aligned");
        launch_jpeg_single(in, rows, cols, quality, coefs, lohi, deq, (long long*)nnz, (cudaStream_t)stream);
    });
}

}  // extern "C"
