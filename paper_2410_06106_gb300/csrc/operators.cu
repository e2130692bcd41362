// Discrete parallel-beam x-ray transform on GB300 (sm_103a):
//   - host-built per-angle tables (int64 fixed-point positions, trapezoid
//     constants) in device memory, copied into shared memory ahead of use,
//   - the ray-driven projector (image chunks staged in shared memory),
//   - the pixel-driven matched backprojector (sinogram windows staged in
//     shared memory) with a plain epilogue and the fused Algorithm 2 u-step,
//   - the C ABI of tomo_geometry_*, tomo_project, tomo_backproject,
//     tomo_opnorm_sq.
//
// The operator (Sec. 2.1, Eq. 2-4): P[(a,b),(i,j)] is the length of the line
// x cos(theta_a) + y sin(theta_a) = t_b inside pixel (i, j). Projected onto
// the ray normal, a unit square is a trapezoid of area 1: with c = cos,
// s = sin, tau = t_b - (x_j c + y_i s),
//   T(tau) = h * sat(0.5 + gamma (w_mid - |tau|)),
//   h = 1/max(|c|,|s|), gamma = 1/min(|c|,|s|), w_mid = max(|c|,|s|)/2.
// For axis-aligned rays (min = 0) gamma is capped at 2^20; every quantity is
// then an exact half-integer, so the formula yields the exact box values
// {1, 1/2, 0} with 1/2 for a ray on a pixel edge.
//
// Both kernels evaluate that same formula, so the backprojector is the exact
// transpose of the projector up to FP32 rounding. Positions are carried in
// 2^-40 fixed point (int64) from the block origin, so that FP32 only ever
// holds offsets below 64 pixels: the weight error stays at ~1e-6 even at
// N = 2048 and for the steep ramps of near-axis angles.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <cudaTypedefs.h>

#include "tomo_internal.cuh"

namespace tomo {

// ------------------------------------------------------------------
// errors
// ------------------------------------------------------------------
static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }
void clear_last_error() { g_last_error.clear(); }
void fail(tomo_status code, const std::string& msg) { throw Error{code, msg}; }

Geometry* as_geometry(tomo_geometry_t g) {
    TOMO_REQUIRE(g != nullptr, "geometry handle is NULL");
    return reinterpret_cast<Geometry*>(g);
}

void check_device(const Geometry& g) {
    int dev = -1;
    TOMO_CUDA(cudaGetDevice(&dev));
    TOMO_REQUIRE(dev == g.device, "geometry was created on device " + std::to_string(g.device) +
                                      " but the current device is " + std::to_string(dev));
}

// ------------------------------------------------------------------
// per-angle parameters: derived on the host in FP64 (tables per geometry)
// ------------------------------------------------------------------
constexpr float kGammaCap = 1048576.0f;  // 2^20
constexpr int kFracBits = 25;
constexpr double kFix25 = (double)(1 << kFracBits);  // 2^25: fixed point of positions inside a block

// 1 + (fraction of a 2^-25 fixed-point position) as a float in [1, 2): the
// top 23 of the 25 fraction bits become the mantissa (exact for the
// half-integer positions of axis-aligned rays)
__device__ __forceinline__ float one_plus_frac25(int p) {
    return __int_as_float(((p >> (kFracBits - 23)) & 0x7FFFFF) | 0x3F800000);
}

// Weights of the two candidate pixels/bins around a position with fraction
// f = F - 1 (distance to the lower candidate, in minor units): the trapezoid
// h sat(0.5 + g (w_mid - dist)) with g the slope in those units gives
//   w_lower = sat(wf0 - g F), w_upper = sat(wf1 + g F),
//   wf0 = 0.5 + g (w_mid + 1), wf1 = 0.5 + g (w_mid - 2).

// host: projector constants of one angle (FP64, then fixed point / FP32)
static ProjAngle make_proj_angle(int N, int B, double c, double s) {
    const double hN = 0.5 * (N - 1), hB = 0.5 * (B - 1);
    const double ac = std::fabs(c), as = std::fabs(s);
    ProjAngle r{};
    double db, dm, k0, maj, mnr;
    if (ac >= as) {  // ray crosses each row once: column coordinate per row
        db = 1.0 / c;
        dm = s / c;
        k0 = -hB / c - (hN * s) / c + hN;
        maj = ac;
        mnr = as;
        r.colmaj = 0;
    } else {  // ray crosses each column once: row coordinate per column
        db = -1.0 / s;
        dm = c / s;
        k0 = hN + hB / s - (hN * c) / s;
        maj = as;
        mnr = ac;
        r.colmaj = 1;
    }
    r.Db = std::llrint(db * kFix);
    r.Dm = std::llrint(dm * kFix);
    r.K0 = std::llrint(k0 * kFix);
    r.dm25 = (int)std::llrint(dm * kFix25);
    const double kap = mnr > 0.0 ? maj / mnr : (double)kGammaCap;
    r.kappa = (float)kap;
    r.wf0 = (float)(0.5 + kap * 1.5);
    r.wf1 = (float)(0.5 - kap * 1.5);
    r.h = (float)(1.0 / maj);
    return r;
}

// host: backprojector constants of one angle
static BpConst make_bp_const(int N, int B, double c, double s) {
    const double hN = 0.5 * (N - 1), hB = 0.5 * (B - 1);
    const double ac = std::fabs(c), as = std::fabs(s);
    const double mx = std::fmax(ac, as), mn = std::fmin(ac, as);
    BpConst r{};
    r.C = std::llrint(c * kFix);
    r.S = std::llrint(s * kFix);
    r.K = std::llrint((hB - hN * c + hN * s) * kFix);
    r.C25 = (int)std::llrint(c * kFix25);
    r.S25 = (int)std::llrint(s * kFix25);
    r.CX16 = (int)std::llrint(16.0 * c * kFix25);
    r.SY8 = (int)std::llrint(8.0 * s * kFix25);
    const double gam = mn > 0.0 ? 1.0 / mn : (double)kGammaCap;
    r.gam = (float)gam;
    r.wf0 = (float)(0.5 + gam * (0.5 * mx + 1.0));
    r.wf1 = (float)(0.5 + gam * (0.5 * mx - 2.0));
    r.h = (float)(1.0 / mx);
    return r;
}

// one angle of a backprojector chunk, for the chunk's tile
// (32 bytes: the inner loop reads it with two 16-byte shared loads)
struct __align__(16) BpAngle {
    unsigned P0;    // bin coordinate of the tile's first pixel minus w0 (2^-25)
    int C25, S25;   // steps of one pixel in x and y (2^-25)
    float gam, wf0, wf1;
    int CX16, SY8;  // steps of 16 pixels in x and 8 in y, rounded once (not rounded single steps)
};

// what the copies of a chunk's windows need per angle
struct BpWin {
    const float* row;  // sinogram line
    int w0;            // first staged bin of this tile
    float h;           // 1 / max(|c|, |s|): applied to the staged window unless the line is prescaled
};

// tile origin (x0, y0), tile extent tw x kBpTileY: the lowest bin
// coordinate over the tile is at the corner picked by the signs of C and S
__device__ __forceinline__ void bp_tile_angle(BpAngle& r, BpWin& wv, const BpConst& k, int x0, int y0, int tw) {
    const long long j = x0 + (k.C < 0 ? tw - 1 : 0);
    const long long i = y0 + (k.S > 0 ? kBpTileY - 1 : 0);
    const long long lo = j * k.C - i * k.S + k.K;
    const int w0 = (int)(lo >> 40) - 2;
    const long long org = (long long)x0 * k.C - (long long)y0 * k.S + k.K;
    r.P0 = (unsigned)((org - ((long long)w0 << 40)) >> (40 - kFracBits));
    r.C25 = k.C25;
    r.S25 = k.S25;
    r.gam = k.gam;
    r.wf0 = k.wf0;
    r.wf1 = k.wf1;
    r.CX16 = k.CX16;
    r.SY8 = k.SY8;
    wv.w0 = w0;
    wv.h = k.h;
}

// asynchronous 4-byte global -> shared copy; zero-fill when !valid
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

// asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ---- TMA (cp.async.bulk.tensor) and mbarrier helpers ---------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"((unsigned)__cvta_generic_to_shared(bar)),
                 "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// one thread: arm the barrier for count boxes of `bytes` each and start their
// 3-D loads: box k from image z + k z_step into dst + k dst_step floats
__device__ __forceinline__ void tma_load_boxes(float* dst, int dst_step, const CUtensorMap* map, int x, int y, int z,
                                               int z_step, int count, uint64_t* bar, unsigned bytes) {
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(bytes * count) : "memory");
    for (int k = 0; k < count; ++k)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
                (unsigned)__cvta_generic_to_shared(dst + k * dst_step)),
            "l"(map), "r"(x), "r"(y), "r"(z + k * z_step), "r"(b)
            : "memory");
}

// nanoseconds of the GPU's global timer
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for the given phase of a barrier; false when the bound ran
// out: `limit_ns` of global time (checked every 256 polls), or 2^28 polls
// should the timer not advance
constexpr uint64_t kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned phase, uint64_t limit_ns = kWaitLimitNs) {
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    uint64_t t0 = 0;
    for (unsigned it = 0; it < (1u << 28); ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(b), "r"(phase)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 255u) {
            const uint64_t t = global_ns();
            if (it == 255u) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
    return false;
}

// failure-detection self test: one thread waits on a barrier that nothing
// arrives at, with the projector's bounded wait; when the bound runs out it
// sets the timeout bit of the status word and returns (no copy is in flight)
__global__ void wait_selftest_kernel(int* status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, limit_ns)) atomicOr(status, 4);
}

// ------------------------------------------------------------------
// projector
// ------------------------------------------------------------------

// thread -> (angle slot, bin offset, row group) of an item:
// na = 4: 4 angles x 128 bins, warp w takes bins 16 (w & 3) .. + 16 of angles
//         2 (w >> 2) and + 1 (half-warps of adjacent angles read nearly the
//         same shared words), and the same bins + 64: two rays per thread
//         (narrow items: 4 angles x 64 bins, one ray per thread);
// na = 2: 2 angles x 128 bins, warp w takes bins 16 w .. + 16 of both;
// na = 1: 128 bins x 2 row groups (threads 128..255 take rows 16..31 of
//         every chunk; the two partial sums are added at the end).
__device__ __forceinline__ void proj_lane_map(int na, int tid, int& slot, int& boff, int& rgrp) {
    const int lane = tid & 31, warp = tid >> 5;
    rgrp = 0;
    if (na == 1) {
        slot = 0;
        boff = tid & 127;
        rgrp = tid >> 7;
    } else if (na == 2) {
        slot = lane >> 4;
        boff = 16 * warp + (lane & 15);
    } else {
        slot = 2 * (warp >> 2) + (lane >> 4);
        boff = 16 * (warp & 3) + (lane & 15);
    }
}


// NR consecutive rows of one ray inside a staged chunk: the two candidate
// pixels of each row, weighted by the trapezoid (see the file header); the
// two candidates accumulate in the two lanes of one packed FP32 pair. With
// PSL slices staged SLF floats apart, the position, weights and address of a
// row serve every slice; tot[s] gathers slice s
template <int NR, int PSL, int SLF>
__device__ __forceinline__ void ray_rows(const float* base, int f0, const ProjAngle& A, float* tot) {
    float2 acc[PSL];
#pragma unroll
    for (int s = 0; s < PSL; ++s) acc[s] = make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int pl = f0 + r * A.dm25;  // position - J at this row (2^-25), may be negative
        const float F = one_plus_frac25(pl);
        const float* t = base + r * kProjPitch + (pl >> kFracBits);  // lower candidate pixel
        const float2 w = make_float2(__saturatef(fmaf(-A.kappa, F, A.wf0)), __saturatef(fmaf(A.kappa, F, A.wf1)));
#pragma unroll
        for (int s = 0; s < PSL; ++s) acc[s] = __ffma2_rn(w, make_float2(t[s * SLF], t[s * SLF + 1]), acc[s]);
    }
#pragma unroll
    for (int s = 0; s < PSL; ++s) tot[s] += acc[s].x + acc[s].y;
}

// two rays of one angle over the same NR rows, interleaved row by row
template <int NR, int PSL, int SLF>
__device__ __forceinline__ void ray_rows2(const float* base0, int f0, const float* base1, int f1, const ProjAngle& A,
                                          float* tot0, float* tot1) {
    float2 acc0[PSL], acc1[PSL];
#pragma unroll
    for (int s = 0; s < PSL; ++s) acc0[s] = acc1[s] = make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int p0 = f0 + r * A.dm25, p1 = f1 + r * A.dm25;
        const float F0 = one_plus_frac25(p0), F1 = one_plus_frac25(p1);
        const float* t0 = base0 + r * kProjPitch + (p0 >> kFracBits);
        const float* t1 = base1 + r * kProjPitch + (p1 >> kFracBits);
        const float2 w0 = make_float2(__saturatef(fmaf(-A.kappa, F0, A.wf0)), __saturatef(fmaf(A.kappa, F0, A.wf1)));
        const float2 w1 = make_float2(__saturatef(fmaf(-A.kappa, F1, A.wf0)), __saturatef(fmaf(A.kappa, F1, A.wf1)));
#pragma unroll
        for (int s = 0; s < PSL; ++s) {
            acc0[s] = __ffma2_rn(w0, make_float2(t0[s * SLF], t0[s * SLF + 1]), acc0[s]);
            acc1[s] = __ffma2_rn(w1, make_float2(t1[s * SLF], t1[s * SLF + 1]), acc1[s]);
        }
    }
#pragma unroll
    for (int s = 0; s < PSL; ++s) {
        tot0[s] += acc0[s].x + acc0[s].y;
        tot1[s] += acc1[s].x + acc1[s].y;
    }
}

// staged minor ranges of chunks c0 .. c0 + 31 of the item (warp 0, lane L:
// chunk c0 + L), written to the ring q0r[chunk & 63]: the first staged column
// (16-byte aligned) from the lowest corner position over the item's angles;
// an extent beyond the stage sets *bad (unreachable: the host bounds it)
template <int R>
__device__ __forceinline__ void proj_q0_batch(const ProjAngle* sa, int na, int b0, int blast, int m_lo, int c0,
                                              int nch, int lane, int* q0r, int* bad) {
    const int c = c0 + lane;
    if (c >= nch) return;
    const long long m0 = m_lo + c * R, m1 = m0 + R - 1;
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (int a = 0; a < na; ++a) {
        const ProjAngle& C = sa[a];
        const long long pb0 = (long long)b0 * C.Db, pb1 = (long long)blast * C.Db;
        const long long pm0 = m0 * C.Dm, pm1 = m1 * C.Dm;
        lo = min(lo, min(pb0, pb1) + min(pm0, pm1) + C.K0);  // the corners are separable in b and m
        hi = max(hi, max(pb0, pb1) + max(pm0, pm1) + C.K0);
    }
    const int q0 = ((int)(lo >> 40) - 2) & ~3;
    q0r[c & 63] = q0;
    if ((int)(hi >> 40) + 3 - q0 > kProjWMax + 3) atomicOr(bad, 1);
}

// PSL slices per item (1, 2 or 4 slices of one node whose rays share the
// position, weight and address arithmetic; chunks of R = kProjRows / PSL rows,
// the stages hold both slices' bands, SLF floats apart)
template <int PSL>
__global__ void __launch_bounds__(kProjThreads, 3) project_kernel(const __grid_constant__ ProjParams p) {
    constexpr int R = kProjRows / PSL;
    constexpr int SLF = R * kProjPitch;
    static_assert(PSL * SLF == kProjStageFloats, "a stage holds PSL bands");
    extern __shared__ __align__(1024) unsigned char proj_dyn[];
    float* stage = reinterpret_cast<float*>(proj_dyn);  // [2][PSL][R][kProjPitch]
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ ProjAngle sa[kProjMaxNa];
    __shared__ int s_item, s_q0[64], s_bad;  // s_q0: staged range per chunk, a ring of 64
    __shared__ float s_part[PSL][kProjThreads / 2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = p.N, B = p.B;
    const size_t n = (size_t)N * N;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
        s_bad = 0;
    }
    __syncthreads();
    unsigned uses0 = 0, uses1 = 0;  // completed loads per stage: the parity to wait for

    for (int pass = 0;; ++pass) {
        int it;
        if (p.counter) {
            if (tid == 0) s_item = atomicAdd(p.counter, 1);
            __syncthreads();
            it = s_item;
        } else {
            it = pass == 0 ? (int)blockIdx.x : p.n_items;
        }
        if (it >= p.n_items || s_bad) break;
        const ProjItem item = p.items[it];
        if (tid < item.na) sa[tid] = p.ptab[p.angs[item.ang0 + tid].angle];
        __syncthreads();

        const int na = item.na;
        int slot, boff, rgrp;
        proj_lane_map(na, tid, slot, boff, rgrp);
        const int b = item.b0 + boff;
        const int blast = min(item.b0 + item.nb - 1, B - 1);
        const int bc = min(b, blast);          // rays past the last bin shadow it (their output is dropped)
        const bool two = na == 4 && item.nb == 128;  // a second ray, 64 bins further
        const int b2 = b + 64, bc2 = min(b2, blast);
        const ProjAngle A = sa[slot];
        const int colmaj = sa[0].colmaj;
        const bool tma = (colmaj ? p.has_mapT : p.has_map) && p.map_rows == R;  // else cp.async staging
        const CUtensorMap* map = colmaj ? &p.mapT : &p.map;
        const float* img = p.img + (size_t)item.img * n;
        // this ray's position at the first row of its row group in chunk 0
        const int r0 = rgrp * (R / 2);
        long long pos = (long long)bc * A.Db + (long long)(item.m_lo + r0) * A.Dm + A.K0;
        long long pos2 = (long long)bc2 * A.Db + (long long)(item.m_lo + r0) * A.Dm + A.K0;
        const long long dpos = (long long)R * A.Dm;
        const int nch = item.nchunks * PSL;  // item.nchunks counts kProjRows-row chunks
        float total[PSL], total2[PSL];
#pragma unroll
        for (int s = 0; s < PSL; ++s) total[s] = total2[s] = 0.f;

        if (warp == 0 && nch > 0) {  // ranges of chunks 0..31; chunk 0's loads when TMA is available
            proj_q0_batch<R>(sa, na, item.b0, blast, item.m_lo, 0, nch, lane, s_q0, &s_bad);
            __syncwarp();
            if (lane == 0 && tma) {
                fence_proxy_async();
                tma_load_boxes(stage, SLF, map, s_q0[0], item.m_lo, item.img, p.pair_img, PSL, &bars[0], 4 * SLF);
            }
        }
        for (int ch = 0; ch < nch; ++ch, pos += dpos, pos2 += dpos) {
            const int sb = ch & 1;
            float* tile = stage + sb * kProjStageFloats;
            const int m0 = item.m_lo + ch * R;
            __syncthreads();  // chunk ch-1 consumed by every thread; s_q0[ch & 63] visible
            if (s_bad) break;
            if (warp == 0 && ch + 1 < nch) {  // next chunk: (TMA) loads into the other stage
                if (((ch + 1) & 31) == 0) {  // ranges of the next 32 chunks (entries 32 back are done)
                    proj_q0_batch<R>(sa, na, item.b0, blast, item.m_lo, ch + 1, nch, lane, s_q0, &s_bad);
                    __syncwarp();
                }
                if (lane == 0 && tma) {
                    fence_proxy_async();
                    tma_load_boxes(stage + (sb ^ 1) * kProjStageFloats, SLF, map, s_q0[(ch + 1) & 63], m0 + R,
                                   item.img, p.pair_img, PSL, &bars[sb ^ 1], 4 * SLF);
                }
            }
            const int q0 = s_q0[ch & 63];
            if (tma) {
                const unsigned ph = sb ? (uses1++ & 1u) : (uses0++ & 1u);
                if (!mbar_wait(&bars[sb], ph)) {  // a load that never lands: give up on the launch
                    if (p.status) atomicOr(p.status, 4);
                    atomicOr(&s_bad, 1);
                }
            } else {
                // cp.async staging of the band (zero outside the image)
                if (!colmaj) {
                    const int ng = kProjPitch / 4;
                    const bool vec = (N & 3) == 0;
                    for (int e = warp; e < PSL * R; e += kProjThreads / 32) {
                        const int sl = e / R, r = e - sl * R;
                        const int row = m0 + r;
                        const bool rok = (unsigned)row < (unsigned)N;
                        const float* simg = img + (size_t)sl * p.pair_img * n;
                        const float* src = simg + (size_t)(rok ? row : 0) * N;
                        float* dst = tile + sl * SLF + r * kProjPitch;
                        for (int g = lane; g < ng; g += 32) {
                            const int col = q0 + 4 * g;
                            if (vec && rok && col >= 0 && col + 4 <= N) {
                                cp_async16(dst + 4 * g, src + col);
                            } else {
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const bool ok = rok && (unsigned)(col + e) < (unsigned)N;
                                    cp_async4(dst + 4 * g + e, ok ? src + col + e : simg, ok);
                                }
                            }
                        }
                    }
                } else if (lane < R) {
                    const int col = m0 + lane;
                    const bool cok = (unsigned)col < (unsigned)N;
#pragma unroll
                    for (int sl = 0; sl < PSL; ++sl) {
                        const float* simg = img + (size_t)sl * p.pair_img * n;
                        for (int q = warp; q < kProjPitch; q += kProjThreads / 32) {
                            const int row = q0 + q;
                            const bool ok = cok && (unsigned)row < (unsigned)N;
                            cp_async4(tile + sl * SLF + lane * kProjPitch + q, ok ? simg + (size_t)row * N + col : simg,
                                      ok);
                        }
                    }
                }
                cp_async_wait_all();
                __syncthreads();
            }
            if (s_bad) continue;  // skip the compute; the loop top exits
            // this ray: integer part J and 2^-25 fraction of its position at its first row
            const int J = (int)(pos >> 40);
            const int f0 = (int)((pos >> (40 - kFracBits)) & ((1 << kFracBits) - 1));
            const float* base = tile + r0 * kProjPitch + (J - q0);
            if (two) {
                const int J2 = (int)(pos2 >> 40);
                const int f2 = (int)((pos2 >> (40 - kFracBits)) & ((1 << kFracBits) - 1));
                ray_rows2<R, PSL, SLF>(base, f0, tile + (J2 - q0), f2, A, total, total2);
            } else if (na == 1) {
                ray_rows<R / 2, PSL, SLF>(base, f0, A, total);
            } else {
                ray_rows<R, PSL, SLF>(base, f0, A, total);
            }
        }
        if (s_bad) {  // wait (bounded) for a load still in flight before leaving
            if (tid == 0 && tma) {
                mbar_wait(&bars[0], uses0 & 1u);
                mbar_wait(&bars[1], uses1 & 1u);
            }
            break;
        }
        if (na == 1) {  // add the second row group's partial sums, in a fixed order
            __syncthreads();
#pragma unroll
            for (int s = 0; s < PSL; ++s)
                if (rgrp) s_part[s][tid & 127] = total[s];
            __syncthreads();
#pragma unroll
            for (int s = 0; s < PSL; ++s)
                if (!rgrp) total[s] += s_part[s][tid];
        }
        if (b < B && !rgrp) {
            const AngRow ar = p.angs[item.ang0 + slot];
#pragma unroll
            for (int s = 0; s < PSL; ++s) {
                const size_t o = ((size_t)item.outb + (size_t)s * p.pair_rows + ar.row) * B + b;
                float v = A.h * total[s];
                if (p.sub) v -= __ldg(p.sub + o);
                if (p.prescale) v *= A.h;
                p.out[o] = v;
                if (two && b2 < B) {
                    float v2 = A.h * total2[s];
                    if (p.sub) v2 -= __ldg(p.sub + o + 64);
                    if (p.prescale) v2 *= A.h;
                    p.out[o + 64] = v2;
                }
            }
        }
        __syncthreads();  // sa / s_item / s_q0 reused by the next item
    }
}

// ------------------------------------------------------------------
// backprojector
// ------------------------------------------------------------------
enum { EPI_STORE = 0, EPI_USTEP = 1 };

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int NPENDING>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NPENDING) : "memory");
}

// asynchronous copies of a chunk's windows: win[a][k] = (r[w0 + k], r[w0 + k + 1])
// of the line, zero outside [0, B); warp w takes angles w, w + 8, ...
// the windows of a chunk's nac angles for SL slices: slice s's window of angle
// a at win + (s CH + a) kBpWin, its line `row_step` floats after slice 0's
template <int SL, int CH, int NT>
__device__ __forceinline__ void bp_issue_windows(float2* win, const BpWin* wv, int nac, int B, size_t row_step,
                                                 int tid) {
    static_assert(kBpWin == 96, "three pairs per lane");
    const int lane = tid & 31;
    for (int e = tid >> 5; e < SL * nac; e += NT / 32) {
        const int sl = SL == 1 ? 0 : e / nac, a = SL == 1 ? e : e - sl * nac;
        const int w0 = wv[a].w0;
        const float* row = wv[a].row + sl * row_step;
        float* d = reinterpret_cast<float*>(win + (sl * CH + a) * kBpWin);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int k = lane + 32 * q, b = w0 + k;
            const bool v0 = (unsigned)b < (unsigned)B, v1 = (unsigned)(b + 1) < (unsigned)B;
            cp_async4(d + 2 * k, v0 ? row + b : row, v0);
            cp_async4(d + 2 * k + 1, v1 ? row + b + 1 : row, v1);
        }
    }
}

__device__ __forceinline__ void prefetch_l2(const void* ptr) {
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(ptr));
}

// Persistent backprojector. A block takes work items from the queue and walks
// their angles in chunks of 32. Everything a chunk needs arrives by cp.async
// ahead of use, so no global latency sits between two chunks: while chunk i
// accumulates, the windows of chunk i + 1, the per-angle constants of chunk
// i + 2 and the descriptor of the item three items ahead are in flight, and
// the queue has already been asked for the item after that. An item's
// epilogue (Algorithm 2 step or store) overlaps the next chunk's copies.
// 16 x 8 threads; thread (tx, ty) owns the PX x 8 pixels (x0 + tx + 16 kx,
// y0 + ty + 8 ky) of a (16 PX) x 64 tile (PX = 4: 64 x 64 tiles; PX = 2:
// 32 x 64 tiles, twice the items for problems with few of them): a half-warp
// (16 consecutive tx) reads 16 window pairs within 16 consecutive entries, so
// its 64-bit shared loads never conflict. A pixel's two candidate bins
// accumulate in the two lanes of one packed FP32 pair (one __ffma2_rn per
// pixel and angle), added together in the epilogue; 8 PX pixels per thread
// spread the per-angle setup over more updates.
// threads of a block: 16 x 8, or 16 x 16 for slice pairs (more warps to cover
// their shorter chunks); RPT rows of pixels per thread
__host__ __device__ constexpr int bp_threads(int slices) { return slices == 2 ? 256 : kBpThreads; }

template <int EPI, int PX, int SL>
__global__ void __launch_bounds__(bp_threads(SL), SL == 2 ? (PX == 4 ? 2 : 3) : 4) backproject_kernel(const BpParams p) {
    constexpr int NT = bp_threads(SL);
    constexpr int TY = NT / 16;          // thread rows
    constexpr int RPT = kBpTileY / TY;   // pixel rows per thread (8, or 4 for slice pairs)
    constexpr int TX = 16 * PX;          // tile width
    constexpr int CH = kBpChunk;         // angles per chunk
    constexpr int STG = SL * CH * kBpWin;  // float2 of a stage: SL windows per angle (24 KB per slice)
    extern __shared__ __align__(16) unsigned char bp_dyn[];
    float2* wins = reinterpret_cast<float2*>(bp_dyn);  // [2][SL][CH][kBpWin]
    __shared__ BpConst s_k[CH];                        // constants of the chunk after next
    __shared__ BpAngle s_a[2][CH];                     // this chunk and the next, for their tiles
    __shared__ BpWin s_w[2][CH];
    const size_t row_step = (size_t)p.pair_rows * p.B;  // second slice's sinogram lines
    __shared__ BpItem s_d[4];                          // descriptors of the block's items j .. j + 3
    __shared__ int s_idx[4];                           // their queue indices (>= n_items: none)
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int N = p.N, B = p.B;
    const size_t n = (size_t)N * N;
    const int n_items = p.n_items;

    auto take = [&]() -> int { return p.counter ? atomicAdd(p.counter, 1) : n_items; };
    auto issue_desc = [&](int slot, int idx) {
        if (tid < 2 && idx < n_items)
            cp_async16(reinterpret_cast<float*>(&s_d[slot]) + 4 * tid,
                       reinterpret_cast<const float*>(p.items + idx) + 4 * tid);
    };
    auto issue_consts = [&](const BpItem& it, int a0) {
        const int nac = min(CH, it.na - a0);
        if (tid < 4 * nac)
            cp_async16(reinterpret_cast<float*>(&s_k[tid >> 2]) + 4 * (tid & 3),
                       reinterpret_cast<const float*>(p.bk + it.ang0 + a0 + (tid >> 2)) + 4 * (tid & 3));
    };
    auto setup = [&](const BpItem& it, int a0, int slot) {
        if (tid < min(CH, it.na - a0)) {
            bp_tile_angle(s_a[slot][tid], s_w[slot][tid], s_k[tid], it.tx * TX, it.ty * kBpTileY, TX);
            s_w[slot][tid].row = p.sino + ((size_t)it.sinb + s_k[tid].row) * B;
        }
    };

    // prologue: queue indices of items 0..2 (and 3, held by thread 0), their
    // descriptors, constants and windows of chunk 0, constants of chunk 1
    int pending = n_items;  // thread 0: queue index of the item three ahead of the current one
    if (tid == 0) {
        int q[3];
        q[0] = p.counter ? atomicAdd(p.counter, 1) : (int)blockIdx.x;
        q[1] = take();
        q[2] = take();
        pending = take();
#pragma unroll
        for (int i = 0; i < 3; ++i) s_idx[i] = q[i];
        s_idx[3] = n_items;
    }
    __syncthreads();
    if (s_idx[0] >= n_items) return;
    for (int i = 0; i < 3; ++i) issue_desc(i, s_idx[i]);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    issue_consts(s_d[0], 0);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    setup(s_d[0], 0, 0);
    __syncthreads();
    int j = 0, a0 = 0, buf = 0;  // the current chunk: item ordinal j, first angle a0
    {
        const BpItem it = s_d[0];
        bp_issue_windows<SL, CH, NT>(wins, s_w[0], min(CH, it.na), B, row_step, tid);
        if (CH < it.na) issue_consts(it, CH);
        else if (s_idx[1] < n_items) issue_consts(s_d[1], 0);
        cp_async_commit();
    }
    float2 acc2[SL][RPT][PX];
#pragma unroll
    for (int sl = 0; sl < SL; ++sl)
#pragma unroll
        for (int ky = 0; ky < RPT; ++ky)
#pragma unroll
            for (int kx = 0; kx < PX; ++kx) acc2[sl][ky][kx] = make_float2(0.f, 0.f);

    for (;;) {
        cp_async_wait<0>();
        __syncthreads();  // (A) windows of this chunk, constants of the next, descriptors up to j + 2 landed
        const BpItem cur = s_d[j & 3];
        const int nac = min(CH, cur.na - a0);
        // the next two chunks of the stream
        int j1 = j, a1 = a0 + CH;
        if (a1 >= cur.na) {
            j1 = j + 1;
            a1 = 0;
        }
        const bool v1 = s_idx[j1 & 3] < n_items;
        const BpItem it1 = s_d[j1 & 3];
        int j2 = j1, a2 = a1 + CH;
        if (v1 && a2 >= it1.na) {
            j2 = j1 + 1;
            a2 = 0;
        }
        const bool v2 = v1 && s_idx[j2 & 3] < n_items;
        if (!p.prescaled) {  // fold h into the pairs this thread copied (its own copies have landed)
            for (int e = tid >> 5; e < SL * nac; e += NT / 32) {
                const int sl = SL == 1 ? 0 : e / nac, a = SL == 1 ? e : e - sl * nac;
                const float h = s_w[buf][a].h;
                float2* w = wins + buf * STG + (sl * CH + a) * kBpWin;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float2 v = w[(tid & 31) + 32 * q];
                    w[(tid & 31) + 32 * q] = make_float2(h * v.x, h * v.y);
                }
            }
        }
        if (v1) setup(it1, a1, buf ^ 1);
        __syncthreads();  // (B) the next chunk's angles are set; the constants slot is free
        if (v1) bp_issue_windows<SL, CH, NT>(wins + (buf ^ 1) * STG, s_w[buf ^ 1], min(CH, it1.na - a1), B, row_step, tid);
        if (v2) issue_consts(s_d[j2 & 3], a2);
        if (a0 == 0 && tid < 32) {  // a new item: the descriptor three items ahead, one more queue index
            const int slot = (j + 3) & 3;
            int idx = 0;
            if (tid == 0) {
                idx = pending;  // taken one item ago, so the queue's latency is hidden
                s_idx[slot] = idx;
                pending = idx < n_items ? take() : n_items;
            }
            issue_desc(slot, __shfl_sync(0xffffffffu, idx, 0));
        }
        cp_async_commit();
        if (EPI == EPI_USTEP && a0 + CH >= cur.na) {
            // the epilogue follows this chunk: bring its rows of u and w into L2 now
            // (one 128-byte line per 32 pixels of a row; a hint, no data moves to
            // registers), so that its loads do not wait on DRAM
            constexpr int LPR = TX / 32;  // lines per tile row
            static_assert(NT >= SL * LPR * kBpTileY, "one thread per line");
            const int sl = tid / (LPR * kBpTileY), t = tid - sl * (LPR * kBpTileY);
            const int row = cur.ty * kBpTileY + t / LPR;
            const int col = cur.tx * TX + 32 * (t % LPR);
            if (tid < SL * LPR * kBpTileY && row < N && col < N) {
                const size_t o = (size_t)(cur.img + sl * p.pair_img) * n + (size_t)row * N + col;
                prefetch_l2(p.view.u + o);
                prefetch_l2(p.view.w + o);
            }
        }

        const float2* win = wins + buf * STG;
        const BpAngle* sab = s_a[buf];
        for (int a = 0; a < nac; ++a) {
            const BpAngle& A = sab[a];
            const float2* wa = win + a * kBpWin;
            const float gam = A.gam, wf0 = A.wf0, wf1 = A.wf1;
            // position - w0 of pixel (x0 + tx, y0 + ty), 2^-25 (non-negative in the tile)
            // row ty + TY ky = (ty & 7) + 8 (ty >> 3 + (TY / 8) ky): the same integer positions
            // (steps of one row and of 8 rows) whatever the block's thread rows
            const unsigned pb = A.P0 + (unsigned)(tx * A.C25) - (unsigned)((ty & 7) * A.S25) -
                                (unsigned)((ty >> 3) * A.SY8);
            const unsigned cx = (unsigned)A.CX16, sy = (unsigned)(TY / 8) * (unsigned)A.SY8;
#pragma unroll
            for (int ky = 0; ky < RPT; ++ky) {
                const unsigned prow = pb - (unsigned)ky * sy;
#pragma unroll
                for (int kx = 0; kx < PX; ++kx) {
                    const unsigned pp = prow + (unsigned)kx * cx;
                    const float F = one_plus_frac25((int)pp);
                    const float2* rp = wa + (pp >> kFracBits);  // (lower bin, upper bin) of slice 0
                    const float2 wgt = make_float2(__saturatef(fmaf(-gam, F, wf0)), __saturatef(fmaf(gam, F, wf1)));
#pragma unroll
                    for (int sl = 0; sl < SL; ++sl)  // the same position and weights serve every slice
                        acc2[sl][ky][kx] = __ffma2_rn(wgt, rp[sl * CH * kBpWin], acc2[sl][ky][kx]);
                }
            }
        }

        if (a0 + CH >= cur.na) {  // the item's last chunk: epilogue for every slice of the item
            const int x0 = cur.tx * TX, y0 = cur.ty * kBpTileY;
            float acc[SL][RPT][PX];  // P^T r of each pixel: its two candidate bins added
#pragma unroll
            for (int sl = 0; sl < SL; ++sl)
#pragma unroll
                for (int ky = 0; ky < RPT; ++ky)
#pragma unroll
                    for (int kx = 0; kx < PX; ++kx) {
                        acc[sl][ky][kx] = acc2[sl][ky][kx].x + acc2[sl][ky][kx].y;
                        acc2[sl][ky][kx] = make_float2(0.f, 0.f);
                    }
            if (EPI == EPI_STORE) {
#pragma unroll
                for (int sl = 0; sl < SL; ++sl) {
                    float* img = p.img + (size_t)(cur.img + sl * p.pair_img) * n;
#pragma unroll
                    for (int ky = 0; ky < RPT; ++ky) {
                        const int row = y0 + ty + TY * ky;
                        if (row >= N) continue;
#pragma unroll
                        for (int kx = 0; kx < PX; ++kx) {
                            const int col = x0 + tx + 16 * kx;
                            if (col >= N) continue;
                            float* o = img + (size_t)row * N + col;
                            *o = (p.beta != 0.f ? *o : 0.f) + acc[sl][ky][kx];
                        }
                    }
                }
            } else {
                // Algorithm 2 step: u <- u - eta1 (P^T r + rho (u - x_m^k) + lambda_m^k)
                //                     = u - eta1 (P^T r + rho u + w_m),
                // w_m = lambda_m^k - rho x_m^k being fixed during the inner steps (the dual
                // update writes it). The slices of an item belong to one node. Every load of
                // every slice is issued before any update, so that one latency round serves
                // the whole item; pixels past the image edge load a valid neighbour and are
                // not stored. u, w and u^T stream through L2 once per launch, so they are
                // loaded and stored evict-first (.cs), which leaves L2 to the residual windows
                // that every tile of the node re-reads.
                const BpView& V = p.view;
                const float eta = V.eta1[cur.node];
                float uo[SL][RPT][PX], wo[SL][RPT][PX];
#pragma unroll
                for (int sl = 0; sl < SL; ++sl) {
                    const size_t io = (size_t)(cur.img + sl * p.pair_img) * n;
#pragma unroll
                    for (int ky = 0; ky < RPT; ++ky) {
                        const size_t ro = io + (size_t)min(y0 + ty + TY * ky, N - 1) * N;
#pragma unroll
                        for (int kx = 0; kx < PX; ++kx) {
                            const int col = min(x0 + tx + 16 * kx, N - 1);
                            uo[sl][ky][kx] = __ldcs(V.u + ro + col);
                            wo[sl][ky][kx] = __ldcs(V.w + ro + col);
                        }
                    }
                }
#pragma unroll
                for (int sl = 0; sl < SL; ++sl) {
                    float* u = V.u + (size_t)(cur.img + sl * p.pair_img) * n;
#pragma unroll
                    for (int ky = 0; ky < RPT; ++ky) {
                        const int row = y0 + ty + TY * ky;
#pragma unroll
                        for (int kx = 0; kx < PX; ++kx) {
                            const int col = x0 + tx + 16 * kx;
                            const float uk = uo[sl][ky][kx];
                            acc[sl][ky][kx] = uk - eta * (acc[sl][ky][kx] + fmaf(V.rho, uk, wo[sl][ky][kx]));
                            if (row < N && col < N) __stcs(u + (size_t)row * N + col, acc[sl][ky][kx]);
                        }
                    }
                }

                if (V.uT) {  // the transposed copy read by the projector's steep-ray items
                    // each slice's tile as TX rows of 64 + 4 floats in this chunk's stage (free
                    // once every thread is done with it): rows 16-byte aligned, so that the copy
                    // out moves 16 bytes per load and store, 4 consecutive pixels of a column of u
                    constexpr int TP = kBpTileY + 4;
                    static_assert(kBpTileY == 64 && SL * TX * TP * 4 <= STG * 8, "transpose tiles");
                    static_assert((TX * kBpTileY) % (4 * NT) == 0, "whole float4 rounds");
                    float* T = reinterpret_cast<float*>(wins + buf * STG);
                    __syncthreads();
#pragma unroll
                    for (int sl = 0; sl < SL; ++sl)
#pragma unroll
                        for (int ky = 0; ky < RPT; ++ky)
#pragma unroll
                            for (int kx = 0; kx < PX; ++kx)
                                T[sl * TX * TP + (tx + 16 * kx) * TP + ty + TY * ky] = acc[sl][ky][kx];
                    __syncthreads();
                    const bool vec = (N & 3) == 0;  // rows of u^T 16-byte aligned (y0 is a multiple of 64)
#pragma unroll
                    for (int sl = 0; sl < SL; ++sl) {
                        float* ut = V.uT + (size_t)(cur.img + sl * p.pair_img) * n;
#pragma unroll
                        for (int i = 0; i < TX * kBpTileY / (4 * NT); ++i) {
                            const int e = tid + i * NT;
                            const int cc = e >> 4, rq = 4 * (e & 15);  // column x0 + cc of u, rows y0 + rq .. + 3
                            if (x0 + cc >= N) continue;
                            const float4 v = *reinterpret_cast<const float4*>(T + sl * TX * TP + cc * TP + rq);
                            float* dst = ut + (size_t)(x0 + cc) * N + y0 + rq;
                            if (vec && y0 + rq + 4 <= N) {
                                __stcs(reinterpret_cast<float4*>(dst), v);
                            } else {  // the image's last rows (unreachable while N % 4 == 0)
                                if (y0 + rq < N) dst[0] = v.x;
                                if (y0 + rq + 1 < N) dst[1] = v.y;
                                if (y0 + rq + 2 < N) dst[2] = v.z;
                                if (y0 + rq + 3 < N) dst[3] = v.w;
                            }
                        }
                    }
                }
            }
        }
        if (!v1) break;
        j = j1;
        a0 = a1;
        buf ^= 1;
    }
    cp_async_wait<0>();
}

// out[k][j][i] = in[k][i][j] for nimg images of N x N
__global__ void transpose_kernel(const float* in, float* out, int N, int nimg) {
    __shared__ float t[32][33];
    const int tiles = (N + 31) / 32;
    for (long long b = blockIdx.x; b < (long long)nimg * tiles * tiles; b += gridDim.x) {
        const int k = (int)(b / ((long long)tiles * tiles));
        const int rem = (int)(b - (long long)k * tiles * tiles);
        const int ti = rem / tiles, tj = rem - ti * tiles;
        const float* src = in + (size_t)k * N * N;
        float* dst = out + (size_t)k * N * N;
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int i = ti * 32 + r, j = tj * 32 + threadIdx.x;
            if (i < N && j < N) t[r][threadIdx.x] = src[(size_t)i * N + j];
        }
        __syncthreads();
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int j = tj * 32 + r, i = ti * 32 + threadIdx.x;
            if (i < N && j < N) dst[(size_t)j * N + i] = t[threadIdx.x][r];
        }
        __syncthreads();
    }
}

void launch_transpose(const float* in, float* out, int N, int nimg, cudaStream_t st) {
    const long long tiles = (long long)nimg * ((N + 31) / 32) * ((N + 31) / 32);
    transpose_kernel<<<(int)std::min<long long>(tiles, 152 * 16), dim3(32, 8), 0, st>>>(in, out, N, nimg);
    TOMO_CUDA(cudaGetLastError());
}

// ---- TMA descriptors -------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

bool make_image_map(CUtensorMap* map, const float* base, int N, int nimg, int rows) {
    std::memset(map, 0, sizeof(*map));
    const auto fn = tensor_map_encoder();
    if (!fn || ((uintptr_t)base & 15) || (N & 3) || nimg < 1) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)nimg};
    const cuuint64_t strides[2] = {(cuuint64_t)N * 4, (cuuint64_t)N * N * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kProjPitch, (cuuint32_t)rows, 1};
    const cuuint32_t elem[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, elem,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static size_t proj_smem() { return sizeof(float) * 2 * kProjStageFloats; }

// the dynamic shared-memory opt-in, set once per process before any capture
static void ensure_proj_attr() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(project_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem());
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(project_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem());
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(project_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem());
    });
    TOMO_CUDA(err);
}

void launch_project(const ProjParams& p, int grid, cudaStream_t st, int slices) {
    if (p.n_items == 0) return;
    ensure_proj_attr();
    if (slices == 4)
        project_kernel<4><<<grid, kProjThreads, proj_smem(), st>>>(p);
    else if (slices == 2)
        project_kernel<2><<<grid, kProjThreads, proj_smem(), st>>>(p);
    else
        project_kernel<1><<<grid, kProjThreads, proj_smem(), st>>>(p);
    TOMO_CUDA(cudaGetLastError());
}

// the window stages (48 KB per slice of an item) and the largest shared carveout,
// so that the blocks the launch bounds ask for fit on an SM; set once per process
template <int EPI, int PX, int SL>
static cudaError_t set_bp_attr() {
    cudaError_t e = cudaFuncSetAttribute(backproject_kernel<EPI, PX, SL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SL * kBpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(backproject_kernel<EPI, PX, SL>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

static void ensure_bp_attr() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = set_bp_attr<EPI_STORE, 4, 1>();
        if (err == cudaSuccess) err = set_bp_attr<EPI_USTEP, 4, 1>();
        if (err == cudaSuccess) err = set_bp_attr<EPI_STORE, 2, 1>();
        if (err == cudaSuccess) err = set_bp_attr<EPI_USTEP, 2, 1>();
        if (err == cudaSuccess) err = set_bp_attr<EPI_STORE, 2, 2>();
        if (err == cudaSuccess) err = set_bp_attr<EPI_USTEP, 2, 2>();
        if (err == cudaSuccess) err = set_bp_attr<EPI_STORE, 4, 2>();
        if (err == cudaSuccess) err = set_bp_attr<EPI_USTEP, 4, 2>();
    });
    TOMO_CUDA(err);
}

// the instantiation of a launch shape
template <int EPI>
static const void* bp_kernel_fn(int tile_x, int slices) {
    if (slices == 2)
        return tile_x == kBpTileXNarrow ? (const void*)backproject_kernel<EPI, 2, 2>
                                        : (const void*)backproject_kernel<EPI, 4, 2>;
    return tile_x == kBpTileXNarrow ? (const void*)backproject_kernel<EPI, 2, 1>
                                    : (const void*)backproject_kernel<EPI, 4, 1>;
}

template <int EPI>
static void launch_bp(const BpParams& p, int grid, cudaStream_t st, int tile_x, int slices) {
    if (p.n_items == 0) return;
    ensure_bp_attr();
    if (slices == 2) {
        if (tile_x == kBpTileXNarrow)
            backproject_kernel<EPI, 2, 2><<<grid, bp_threads(2), 2 * kBpSmem, st>>>(p);
        else
            backproject_kernel<EPI, 4, 2><<<grid, bp_threads(2), 2 * kBpSmem, st>>>(p);
    } else if (tile_x == kBpTileXNarrow) {
        backproject_kernel<EPI, 2, 1><<<grid, kBpThreads, kBpSmem, st>>>(p);
    } else {
        backproject_kernel<EPI, 4, 1><<<grid, kBpThreads, kBpSmem, st>>>(p);
    }
    TOMO_CUDA(cudaGetLastError());
}

void launch_backproject_store(const BpParams& p, int grid, cudaStream_t st, int tile_x, int slices) {
    launch_bp<EPI_STORE>(p, grid, st, tile_x, slices);
}

void launch_backproject_ustep(const BpParams& p, int grid, cudaStream_t st, int tile_x, int slices) {
    launch_bp<EPI_USTEP>(p, grid, st, tile_x, slices);
}

static int sm_count() {
    int dev = 0, sms = 0;
    TOMO_CUDA(cudaGetDevice(&dev));
    TOMO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms;
}

int persistent_grid_project(int slices) {
    int per_sm = 0;
    ensure_proj_attr();
    const void* fn = slices == 4   ? (const void*)project_kernel<4>
                     : slices == 2 ? (const void*)project_kernel<2>
                                   : (const void*)project_kernel<1>;
    TOMO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kProjThreads, proj_smem()));
    return sm_count() * (per_sm > 0 ? per_sm : 1);
}

int persistent_grid_backproject(bool ustep, int tile_x, int slices) {
    int per_sm = 0;
    ensure_bp_attr();
    const void* fn = ustep ? bp_kernel_fn<EPI_USTEP>(tile_x, slices) : bp_kernel_fn<EPI_STORE>(tile_x, slices);
    TOMO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, bp_threads(slices), slices * kBpSmem));
    return sm_count() * (per_sm > 0 ? per_sm : 1);
}

// ------------------------------------------------------------------
// host work-list builders
// ------------------------------------------------------------------
namespace {
struct HostProj {  // FP64 mirror of ProjAngle (positions, not fixed point)
    double db, dm, k0;
    bool colmaj;
};
HostProj host_proj(const Geometry& g, int a) {
    const double c = g.c[a], s = g.s[a], hN = 0.5 * (g.N - 1), hB = 0.5 * (g.B - 1);
    HostProj r;
    if (rows_major(c, s)) {
        r.db = 1.0 / c;
        r.dm = s / c;
        r.k0 = -hB / c - (hN * s) / c + hN;
        r.colmaj = false;
    } else {
        r.db = -1.0 / s;
        r.dm = c / s;
        r.k0 = hN + hB / s - (hN * c) / s;
        r.colmaj = true;
    }
    return r;
}

// major-index interval [lo, hi] on which any ray b0..b1 of angle A lies
// within the image's minor range (conservative by one pixel)
void major_range(const HostProj& A, int b0, int b1, int N, int& lo, int& hi) {
    const double plo = std::min(b0 * A.db, b1 * A.db) + A.k0;
    const double phi = std::max(b0 * A.db, b1 * A.db) + A.k0;
    const double lim_lo = -2.0, lim_hi = N + 1.0;
    // need m dm + phi >= lim_lo and m dm + plo <= lim_hi
    double a = 0.0, b = N - 1.0;
    if (A.dm > 0) {
        a = std::max(a, (lim_lo - phi) / A.dm);
        b = std::min(b, (lim_hi - plo) / A.dm);
    } else if (A.dm < 0) {
        a = std::max(a, (lim_hi - plo) / A.dm);
        b = std::min(b, (lim_lo - phi) / A.dm);
    } else if (phi < lim_lo || plo > lim_hi) {
        b = -1.0;
    }
    lo = (int)std::floor(a) - 1;
    hi = (int)std::ceil(b) + 1;
    lo = std::max(lo, 0);
    hi = std::min(hi, N - 1);
}

// upper bound of the staged extent of one item chunk, mirroring the kernel
int chunk_extent(const std::vector<HostProj>& As, int b0, int b1, int m0) {
    double lo = 1e300, hi = -1e300;
    for (const HostProj& A : As)
        for (int bb : {b0, b1})
            for (int mm : {m0, m0 + kProjRows - 1}) {
                const double v = bb * A.db + mm * A.dm + A.k0;
                lo = std::min(lo, v);
                hi = std::max(hi, v);
            }
    const int q0 = (int)std::floor(lo) - 2;
    return (int)std::floor(hi) + 3 - q0 + 2;  // +2 slack over the kernel's fixed-point value
}
}  // namespace

void build_proj_items(const Geometry& g, const std::vector<AngRow>& angs, int ang_begin,
                      int ang_count, int img, int outb, std::vector<ProjItem>& out, int bins4) {
    const int end = ang_begin + ang_count;
    int i = ang_begin;
    while (i < end) {
        int na = kProjMaxNa;
        for (; na >= 1; na /= 2) {
            if (i + na > end) continue;
            const bool cm = rows_major(g.c[angs[i].angle], g.s[angs[i].angle]);
            bool same = true;
            for (int k = 1; k < na; ++k)
                same &= rows_major(g.c[angs[i + k].angle], g.s[angs[i + k].angle]) == cm;
            if (!same) continue;
            // extent check over every bin run and chunk
            std::vector<HostProj> As;
            for (int k = 0; k < na; ++k) As.push_back(host_proj(g, angs[i + k].angle));
            const int wb = na == 4 ? bins4 : kProjItemBins;
            bool ok = true;
            for (int b0 = 0; b0 < g.B && ok; b0 += wb) {
                const int b1 = std::min(b0 + wb - 1, g.B - 1);
                int lo = g.N, hi = -1;
                for (const HostProj& A : As) {
                    int l, h;
                    major_range(A, b0, b1, g.N, l, h);
                    if (h >= l) {
                        lo = std::min(lo, l);
                        hi = std::max(hi, h);
                    }
                }
                for (int m0 = lo; m0 <= hi && ok; m0 += kProjRows)
                    ok = chunk_extent(As, b0, b1, m0) <= kProjWMax;
            }
            if (ok) break;
        }
        if (na < 1)  // cannot happen for the limits checked at geometry creation
            fail(TOMO_ERR_INVALID_ARG, "projector item exceeds the staged extent (angle " +
                                           std::to_string(angs[i].angle) + ")");
        std::vector<HostProj> As;
        for (int k = 0; k < na; ++k) As.push_back(host_proj(g, angs[i + k].angle));
        const int wb = na == 4 ? bins4 : kProjItemBins;
        for (int b0 = 0; b0 < g.B; b0 += wb) {
            const int b1 = std::min(b0 + wb - 1, g.B - 1);
            int lo = g.N, hi = -1;
            for (const HostProj& A : As) {
                int l, h;
                major_range(A, b0, b1, g.N, l, h);
                if (h >= l) {
                    lo = std::min(lo, l);
                    hi = std::max(hi, h);
                }
            }
            ProjItem it{};
            it.img = img;
            it.outb = outb;
            it.ang0 = i;
            it.na = na;
            it.b0 = b0;
            it.m_lo = hi >= lo ? lo : 0;
            it.nchunks = hi >= lo ? ceil_div(hi - lo + 1, kProjRows) : 0;
            it.nb = wb;
            out.push_back(it);
        }
        i += na;
    }
}

std::vector<BpConst> bp_list_consts(const Geometry& g, const std::vector<AngRow>& angs) {
    std::vector<BpConst> out(angs.size());
    for (size_t q = 0; q < angs.size(); ++q) {
        out[q] = g.hb[angs[q].angle];
        out[q].row = angs[q].row;
    }
    return out;
}

void build_bp_items(const Geometry& g, int ang_begin, int ang_count, int img, int sinb, int node,
                    int slice, std::vector<BpItem>& out, int tile_x) {
    const int ntx = ceil_div(g.N, tile_x), nty = ceil_div(g.N, kBpTileY);
    for (int ty = 0; ty < nty; ++ty)
        for (int tx = 0; tx < ntx; ++tx) {
            BpItem it{};
            it.img = img;
            it.sinb = sinb;
            it.tx = tx;
            it.ty = ty;
            it.ang0 = ang_begin;
            it.na = ang_count;
            it.node = node;
            it.slice = slice;
            out.push_back(it);
        }
}

// ------------------------------------------------------------------
// opnorm helpers
// ------------------------------------------------------------------
__global__ void opnorm_init_kernel(float* x, size_t n, uint64_t seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        x[i] = (float)((z >> 40) * (1.0 / 16777216.0));
    }
}

// out[0] = <x, y>, out[1] = <y, y> in FP64 (one block)
__global__ void opnorm_dot_kernel(const float* x, const float* y, size_t n, double* out) {
    __shared__ double s0[32], s1[32];
    double a = 0.0, b = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        a += (double)x[i] * y[i];
        b += (double)y[i] * y[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s0[threadIdx.x >> 5] = a;
        s1[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ta += s0[w];
            tb += s1[w];
        }
        out[0] = ta;
        out[1] = tb;
    }
}

__global__ void opnorm_scale_kernel(const float* y, float* x, size_t n, const double* dots) {
    const float inv = (float)(1.0 / sqrt(dots[1]));
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] = y[i] * inv;
}

}  // namespace tomo

using namespace tomo;

// ------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------
extern "C" {

const char* tomo_last_error(void) { return tomo::g_last_error.c_str(); }

int tomo_version(void) { return 100; }

tomo_status tomo_geometry_create(int N, int n_bins, int n_angles, const double* angles_rad,
                                 tomo_geometry_t* out) {
    return guard([&] {
        TOMO_REQUIRE(out != nullptr, "out is NULL");
        *out = nullptr;
        TOMO_REQUIRE(N >= 1 && N <= 8192, "N must be in [1, 8192]");
        TOMO_REQUIRE(n_bins >= 1 && n_bins <= 16384, "n_bins must be in [1, 16384]");
        TOMO_REQUIRE(n_angles >= 1 && n_angles <= 4096, "n_angles must be in [1, 4096]");
        auto* g = new Geometry();
        g->N = N;
        g->B = n_bins;
        g->A = n_angles;
        g->c.resize(n_angles);
        g->s.resize(n_angles);
        const double half_pi = 1.57079632679489661923;
        std::vector<ProjAngle> pt(n_angles);
        std::vector<BpConst> bt(n_angles);
        for (int a = 0; a < n_angles; ++a) {
            const double th = angles_rad ? angles_rad[a] : a * (3.14159265358979323846 / n_angles);
            if (!std::isfinite(th)) {
                delete g;
                fail(TOMO_ERR_INVALID_ARG, "angle " + std::to_string(a) + " is not finite");
            }
            const double k = std::floor(th / half_pi + 0.5);
            double c, s;
            if (std::fabs(th - k * half_pi) < 1e-12) {
                const long m = (((long)k % 4) + 4) % 4;
                c = m == 0 ? 1.0 : m == 2 ? -1.0 : 0.0;
                s = m == 1 ? 1.0 : m == 3 ? -1.0 : 0.0;
            } else {
                c = std::cos(th);
                s = std::sin(th);
            }
            g->c[a] = c;
            g->s[a] = s;
            pt[a] = make_proj_angle(N, n_bins, c, s);
            bt[a] = make_bp_const(N, n_bins, c, s);
        }
        g->hb = std::move(bt);
        cudaError_t e = cudaGetDevice(&g->device);
        if (e == cudaSuccess) e = cudaMalloc(&g->d_ptab, sizeof(ProjAngle) * n_angles);
        if (e == cudaSuccess) e = cudaMalloc(&g->d_status, sizeof(int) * 4);
        if (e == cudaSuccess) e = cudaMemset(g->d_status, 0, sizeof(int) * 4);
        if (e == cudaSuccess)
            e = cudaMemcpy(g->d_ptab, pt.data(), sizeof(ProjAngle) * n_angles, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(g->d_ptab);
            cudaFree(g->d_status);
            delete g;
            fail(TOMO_ERR_CUDA, std::string("tomo_geometry_create: ") + cudaGetErrorString(e));
        }
        *out = reinterpret_cast<tomo_geometry_t>(g);
    });
}

tomo_status tomo_geometry_destroy(tomo_geometry_t gh) {
    return guard([&] {
        if (!gh) return;
        Geometry* g = as_geometry(gh);
        for (auto& s : g->cache) cudaFree(s.d_block);
        cudaFree(g->d_ptab);
        cudaFree(g->d_status);
        delete g;
    });
}

}  // extern "C"

namespace tomo {
// cached work lists of a standalone selection (angle list + batch): a hit moves
// the entry to the most recent end and allocates nothing; a miss builds the
// lists, copies them into one device allocation and drops least recently used
// entries beyond the budget
static Geometry::Sel& selection(Geometry& g, const int32_t* angle_idx, int n_sel, int batch) {
    std::vector<int32_t> key(n_sel);
    uint64_t h = 1469598103934665603ull ^ (uint64_t)batch;
    for (int q = 0; q < n_sel; ++q) {
        const int a = angle_idx ? angle_idx[q] : q;
        TOMO_REQUIRE(a >= 0 && a < g.A, "angle index " + std::to_string(a) + " out of range");
        key[q] = a;
        h = (h ^ (uint64_t)(uint32_t)a) * 1099511628211ull;
    }
    std::lock_guard<std::mutex> lk(g.mu);
    for (auto it = g.cache.begin(); it != g.cache.end(); ++it)
        if (it->hash == h && it->batch == batch && it->key == key) {
            g.cache.splice(g.cache.end(), g.cache, it);
            return g.cache.back();
        }
    Geometry::Sel s;
    s.key = key;
    s.hash = h;
    s.batch = batch;
    std::vector<AngRow> angs(n_sel);
    for (int q = 0; q < n_sel; ++q) angs[q] = AngRow{key[q], q};
    std::vector<ProjItem> pi;
    std::vector<BpItem> bi;
    for (int k = 0; k < batch; ++k) {
        build_proj_items(g, angs, 0, n_sel, k, k * n_sel, pi);
        build_bp_items(g, 0, n_sel, k, k * n_sel, 0, 0, bi);
    }
    const std::vector<BpConst> bk = bp_list_consts(g, angs);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t o_angs = 0, o_bk = o_angs + al(sizeof(AngRow) * angs.size());
    const size_t o_pi = o_bk + al(sizeof(BpConst) * bk.size());
    const size_t o_bi = o_pi + al(sizeof(ProjItem) * pi.size());
    s.bytes = o_bi + al(sizeof(BpItem) * bi.size());
    std::vector<unsigned char> host(s.bytes, 0);
    std::memcpy(host.data() + o_angs, angs.data(), sizeof(AngRow) * angs.size());
    std::memcpy(host.data() + o_bk, bk.data(), sizeof(BpConst) * bk.size());
    if (!pi.empty()) std::memcpy(host.data() + o_pi, pi.data(), sizeof(ProjItem) * pi.size());
    if (!bi.empty()) std::memcpy(host.data() + o_bi, bi.data(), sizeof(BpItem) * bi.size());
    while (!g.cache.empty() &&
           (g.cache_bytes + s.bytes > kSelCacheBytes || g.cache.size() >= kSelCacheEntries)) {
        cudaFree(g.cache.front().d_block);
        g.cache_bytes -= g.cache.front().bytes;
        ++g.list_frees;
        g.cache.pop_front();
    }
    TOMO_CUDA(cudaMalloc(&s.d_block, s.bytes));
    ++g.list_allocs;
    const cudaError_t e = cudaMemcpy(s.d_block, host.data(), s.bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(s.d_block);
        ++g.list_frees;
        fail(TOMO_ERR_CUDA, std::string("work-list upload: ") + cudaGetErrorString(e));
    }
    unsigned char* base = static_cast<unsigned char*>(s.d_block);
    s.d_angs = reinterpret_cast<AngRow*>(base + o_angs);
    s.d_bk = reinterpret_cast<BpConst*>(base + o_bk);
    s.d_pitems = pi.empty() ? nullptr : reinterpret_cast<ProjItem*>(base + o_pi);
    s.n_pitems = (int)pi.size();
    s.d_bitems = bi.empty() ? nullptr : reinterpret_cast<BpItem*>(base + o_bi);
    s.n_bitems = (int)bi.size();
    g.cache_bytes += s.bytes;
    g.cache.push_back(std::move(s));
    return g.cache.back();
}
}  // namespace tomo

extern "C" {

tomo_status tomo_project(tomo_geometry_t gh, const float* img, float* sino, const int32_t* angle_idx,
                         int n_sel, int batch, const float* subtract, tomo_stream_t stream) {
    return guard([&] {
        Geometry* g = as_geometry(gh);
        check_device(*g);
        TOMO_REQUIRE(img && sino, "img and sino must be non-NULL");
        TOMO_REQUIRE(batch >= 1, "batch must be >= 1");
        TOMO_REQUIRE(n_sel >= 1 && n_sel <= 65536, "n_sel out of range");
        TOMO_REQUIRE(angle_idx || n_sel == g->A, "angle_idx NULL requires n_sel == n_angles");
        Geometry::Sel& s = selection(*g, angle_idx, n_sel, batch);
        ProjParams p{};
        p.has_map = make_image_map(&p.map, img, g->N, batch) ? 1 : 0;
        p.map_rows = kProjRows;
        p.has_mapT = 0;
        p.img = img;
        p.out = sino;
        p.sub = subtract;
        p.items = s.d_pitems;
        p.angs = s.d_angs;
        p.counter = nullptr;
        p.status = g->d_status;
        p.n_items = s.n_pitems;
        p.ptab = g->d_ptab;
        p.N = g->N;
        p.B = g->B;
        p.prescale = 0;
        launch_project(p, s.n_pitems, (cudaStream_t)stream);
    });
}

tomo_status tomo_backproject(tomo_geometry_t gh, const float* sino, float* img, const int32_t* angle_idx,
                             int n_sel, int batch, float beta, tomo_stream_t stream) {
    return guard([&] {
        Geometry* g = as_geometry(gh);
        check_device(*g);
        TOMO_REQUIRE(img && sino, "img and sino must be non-NULL");
        TOMO_REQUIRE(batch >= 1, "batch must be >= 1");
        TOMO_REQUIRE(beta == 0.f || beta == 1.f, "beta must be 0 or 1");
        TOMO_REQUIRE(n_sel >= 1 && n_sel <= 65536, "n_sel out of range");
        TOMO_REQUIRE(angle_idx || n_sel == g->A, "angle_idx NULL requires n_sel == n_angles");
        Geometry::Sel& s = selection(*g, angle_idx, n_sel, batch);
        BpParams p{};
        p.sino = sino;
        p.img = img;
        p.items = s.d_bitems;
        p.bk = s.d_bk;
        p.n_items = s.n_bitems;
        p.N = g->N;
        p.B = g->B;
        p.prescaled = 0;
        p.beta = beta;
        launch_backproject_store(p, s.n_bitems, (cudaStream_t)stream);
    });
}

tomo_status tomo_geometry_plan(tomo_geometry_t gh, const int32_t* angle_idx, int n_sel, int batch) {
    return guard([&] {
        Geometry* g = as_geometry(gh);
        check_device(*g);
        TOMO_REQUIRE(batch >= 1, "batch must be >= 1");
        TOMO_REQUIRE(n_sel >= 1 && n_sel <= 65536, "n_sel out of range");
        TOMO_REQUIRE(angle_idx || n_sel == g->A, "angle_idx NULL requires n_sel == n_angles");
        selection(*g, angle_idx, n_sel, batch);
    });
}

tomo_status tomo_geometry_cache_stats(tomo_geometry_t gh, int64_t* allocs, int64_t* frees, int64_t* entries,
                                      int64_t* bytes) {
    return guard([&] {
        Geometry* g = as_geometry(gh);
        std::lock_guard<std::mutex> lk(g->mu);
        if (allocs) *allocs = g->list_allocs;
        if (frees) *frees = g->list_frees;
        if (entries) *entries = (int64_t)g->cache.size();
        if (bytes) *bytes = (int64_t)g->cache_bytes;
    });
}

size_t tomo_opnorm_workspace_size(tomo_geometry_t gh, int n_sel) {
    if (!gh || n_sel < 1) return 0;
    Geometry* g = reinterpret_cast<Geometry*>(gh);
    const size_t n = (size_t)g->N * g->N;
    return 256 + sizeof(float) * (2 * n + (size_t)n_sel * g->B) + 2 * sizeof(double) + 256;
}

tomo_status tomo_opnorm_sq(tomo_geometry_t gh, const int32_t* angle_idx, int n_sel, int iters,
                           uint64_t seed, void* work, size_t work_bytes, double* out,
                           tomo_stream_t stream) {
    return guard([&] {
        Geometry* g = as_geometry(gh);
        check_device(*g);
        TOMO_REQUIRE(out && work, "out and work must be non-NULL");
        TOMO_REQUIRE(iters >= 1, "iters must be >= 1");
        TOMO_REQUIRE(work_bytes >= tomo_opnorm_workspace_size(gh, n_sel), "workspace too small");
        const size_t n = (size_t)g->N * g->N;
        char* w = (char*)(((uintptr_t)work + 255) & ~(uintptr_t)255);
        float* x = (float*)w;
        float* z = x + n;
        float* y = z + n;
        double* dots = (double*)(((uintptr_t)(y + (size_t)n_sel * g->B) + 15) & ~(uintptr_t)15);
        cudaStream_t st = (cudaStream_t)stream;
        opnorm_init_kernel<<<256, 256, 0, st>>>(x, n, seed);
        TOMO_CUDA(cudaGetLastError());
        // normalise the start vector
        opnorm_dot_kernel<<<1, 1024, 0, st>>>(x, x, n, dots);
        opnorm_scale_kernel<<<256, 256, 0, st>>>(x, x, n, dots);
        for (int it = 0; it < iters; ++it) {
            tomo_status rc = tomo_project(gh, x, y, angle_idx, n_sel, 1, nullptr, stream);
            if (rc != TOMO_OK) fail(rc, tomo_last_error());
            rc = tomo_backproject(gh, y, z, angle_idx, n_sel, 1, 0.f, stream);
            if (rc != TOMO_OK) fail(rc, tomo_last_error());
            opnorm_dot_kernel<<<1, 1024, 0, st>>>(x, z, n, dots);  // <x, P^T P x>, ||P^T P x||^2
            if (it + 1 < iters) opnorm_scale_kernel<<<256, 256, 0, st>>>(z, x, n, dots);
            TOMO_CUDA(cudaGetLastError());
        }
        double h[2];
        TOMO_CUDA(cudaMemcpyAsync(h, dots, sizeof(h), cudaMemcpyDeviceToHost, st));
        TOMO_CUDA(cudaStreamSynchronize(st));
        *out = h[0];  // Rayleigh quotient at the unit vector x
        const tomo_status rc = tomo_sync_status(gh, stream);
        if (rc != TOMO_OK) fail(rc, tomo_last_error());
    });
}

tomo_status tomo_selftest_wait(tomo_geometry_t gh, int timeout_ms, tomo_stream_t stream) {
    return guard([&] {
        Geometry* g = as_geometry(gh);
        check_device(*g);
        TOMO_REQUIRE(timeout_ms >= 1 && timeout_ms <= 2000, "timeout_ms must be in [1, 2000]");
        wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(g->d_status, (uint64_t)timeout_ms * 1000000ull);
        TOMO_CUDA(cudaGetLastError());
    });
}

tomo_status tomo_sync_status(tomo_geometry_t gh, tomo_stream_t stream) {
    return guard([&] {
        Geometry* g = as_geometry(gh);
        check_device(*g);
        cudaStream_t st = (cudaStream_t)stream;
        int status = 0;
        TOMO_CUDA(cudaMemcpyAsync(&status, g->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
        TOMO_CUDA(cudaMemsetAsync(g->d_status, 0, sizeof(int), st));
        TOMO_CUDA(cudaStreamSynchronize(st));
        if (status & 4) fail(TOMO_ERR_TIMEOUT, "a bounded wait for a staged image band gave up; the projection is incomplete");
        if (status & 1) fail(TOMO_ERR_CUDA, "projector staging extent exceeded (internal error)");
    });
}

}  // extern "C"
