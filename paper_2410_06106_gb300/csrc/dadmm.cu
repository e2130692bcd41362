// Decentralized ADMM with quantized messages (Sec. 2.4-2.7, Algorithms 2-4,
// Eq. 15-18 and 21-24) for S independent slices of M simulated nodes on one
// GB300.
//
// One iteration:
//   E1 x [ projector + residual  (persistent kernel over every (slice, node,
//          angle group, bin run) item)
//        | backprojector + fused u-step (persistent kernel over every
//          (slice, node, 64x32 tile) item) ]                 Algorithm 2
//   x-step on every owner's segment + identity messages + segment min/max
//                                                               Algorithm 3
//   K-means messages (one CTA per owner) and JPEG messages      Eq. 23
//   dual update of every node against its view of x + FP64 partial norms
//                                                               Eq. 24
//   statistics and the iteration counter
//
// Message graph (the paper sends every segment to every node, Sec. 2.5;
// here any connected graph): segment s reaches node m along the shortest
// path with lowest-id parents, one hop per iteration, relayed verbatim, so
// node m's view of segment s at iteration k is the message of iteration
// k - max(dist(s,m) - 1, 0) through the quantizer of the path's first edge.
// Messages live in a ring hist[D][kind][S][N][N] that every reader indexes
// with (k - lag) mod D; the iteration counter lives on the device so one
// captured CUDA graph serves every iteration.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <cmath>
#include <numeric>
#include <queue>

#include "tomo_internal.cuh"

namespace tomo {

void prepare_codecs(int km_k);

constexpr int kStatsCap = 1024;   // statistics ring (iterations)
constexpr int kGraphCache = 4;    // captured iterations kept per handle
constexpr int kDualPerNode = 8;   // dual-kernel blocks per (slice, node)
constexpr int kResPerSlice = 64;  // residual-norm blocks per slice
constexpr int kElemThreads = 256;

struct Dadmm {
    Geometry* g = nullptr;
    int N = 0, B = 0, A = 0, S = 0, M = 0, D = 1;
    int E1 = 0, E2 = 0, km_k = 0, km_iters = 0, jpeg_q = 50, mode = 0;
    double rho = 1.0, eta2 = 0.0;
    uint64_t seed = 0;
    std::vector<int32_t> seg_row_ptr, home_q;
    std::vector<int8_t> lag, kind;  // [node][segment]
    std::vector<int32_t> recv_cnt;  // [owner][3]: receivers of each kind
    std::vector<int32_t> need;      // [owner]: bitmask of message kinds produced
    // device tables
    AngRow* d_angs = nullptr;
    ProjItem* d_pitems = nullptr;   // batched order (longest first)
    BpItem* d_bitems = nullptr;
    BpConst* d_bk = nullptr;  // backprojector constants of the node-major angle list
    ProjItem* d_pplain = nullptr;   // grouped by (slice, node)
    BpItem* d_bplain = nullptr;
    int n_pitems = 0, n_bitems = 0;
    std::vector<int> p_range, b_range;  // [(slice*M + node) * 2]: begin, end in the plain lists
    int8_t* d_lag = nullptr;
    int8_t* d_kind = nullptr;
    int32_t* d_seg_of_row = nullptr;
    int32_t* d_need = nullptr;
    int32_t* d_recv = nullptr;
    int32_t* d_home = nullptr;
    float* d_eta1 = nullptr;
    float* d_eta0 = nullptr;  // [M] zeros: the autotuner's u-step trials leave u as it is
    float* d_mx = nullptr;  // [A] max(|cos|, |sin|) per angle: undoes the residual's prescale
    SegTask* d_km = nullptr;
    SegTask* d_jp = nullptr;
    int n_km = 0, n_jp = 0, max_jp_rows = 0;
    std::vector<int> km_slice_begin, jp_slice_begin;  // tasks are slice-major: per-(slice, owner) index
    std::vector<int> km_index, jp_index;              // [(slice*M + owner)] -> task index or -1
    int grid_proj = 0, grid_bp = 0;
    // launch shapes (K9): backprojector tile width, bins of 4-angle projector items;
    // tune: 0 wide shapes, 1 timed at the first step and cached per problem shape,
    // 2 narrow shapes
    int tune = 0, bp_tile_x = kBpTileXWide, proj_bins4 = kProjItemBins;
    int bp_slices = 1;    // batched backprojector items: 1 slice, or 2 slices of one node and tile
    int proj_slices = 1;  // projector items (both forms): 1 slice, or 2 or 4 slices of one node
    int map_rows = kProjRows;  // box height of map_u / map_uT (kProjRows / proj_slices)
    bool tuned = false;
    std::vector<AngRow> angs;           // node-major angle list
    std::vector<int32_t> node_ang_ptr;  // [M + 1]
    // workspace layout (byte offsets from the aligned base)
    size_t off_resid = 0, off_counters = 0, off_lo = 0, off_hi = 0, off_nnz = 0, off_coefs = 0, off_bits = 0, off_dual = 0,
           off_res = 0, off_stats = 0, off_status = 0, off_uT = 0, off_w = 0, ws_bytes = 0;
    const void* ws_status_init = nullptr;  // workspace whose status word this handle has zeroed
    // the workspace's arrays derived from the state (the transposed copy of u, and
    // w = lambda - rho x of every node) are current for (der_u, der_ws) unless der_dirty
    const void* der_u = nullptr;
    const void* der_ws = nullptr;
    bool der_dirty = true;
    // lost messages: versions held [node][segment] after iteration held_k (host), the
    // table of the current lossy call, and whether the captured graph reads it
    int max_stale = 0;
    std::vector<int32_t> held;
    int held_k = -1;
    bool held_stale = false;  // some node held an old version after iteration held_k
    std::vector<int32_t> held_tab;
    bool lossy = false;
    size_t off_held = 0;
    // neighbour-averaged consensus variant: closed neighbourhoods (sender | quantizer << 16)
    int variant = 0;
    int32_t* d_nb_ptr = nullptr;
    int32_t* d_nb = nullptr;
    // TMA descriptors of u and of its transposed copy (rebuilt with the graph)
    CUtensorMap map_u{}, map_uT{};
    int has_maps = 0;
    // stream / graph
    cudaStream_t own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // captured iterations, one per set of state, workspace and input pointers, least
    // recently used first (a caller that alternates a few input buffers does not
    // re-capture)
    struct Captured {
        std::vector<const void*> key;
        cudaGraphExec_t exec;
    };
    std::vector<Captured> graphs;
    void drop_graphs() {
        for (Captured& c : graphs) cudaGraphExecDestroy(c.exec);
        graphs.clear();
    }
    // phase timing
    bool profiling = false;
    std::vector<cudaEvent_t> pev;  // num_phases + 1 boundaries
    int num_phases() const { return 2 * E1 + 5; }
};

static Dadmm* as_dadmm(dadmm_t h) {
    TOMO_REQUIRE(h != nullptr, "dadmm handle is NULL");
    return reinterpret_cast<Dadmm*>(h);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------
struct ElemParams {
    float* u;      // [S][M][N][N]
    float* lam;    // [S][M][N][N]
    float* xseg;   // [S][N][N]
    float* hist;   // [D][3][S][N][N]
    int32_t* iter;
    const int32_t* seg_of_row;
    const int8_t* lag;
    const int8_t* kind;
    const int32_t* held;     // lossy steps: [iteration - *k_first][2][M][M] (null: lag rule)
    const int32_t* k_first;
    const int32_t* need;
    unsigned* lo_key;
    unsigned* hi_key;
    double* dual_part;  // [S][M*kDualPerNode][3]
    float* w;           // [S][M][N][N] written with lambda: lambda_m^{k+1} - rho x_m^{k+1}
    int N, S, M, D, E2;
    float rho, eta2rho, inv_rho;
};

// Algorithm 3 on every row of every owner's segment, E2 steps in registers:
// x <- x - eta2 rho (x - u_m - lambda_m / rho); then the identity message and
// the segment's min / max (JPEG sample map)
__global__ void __launch_bounds__(kElemThreads) xstep_kernel(const ElemParams p, int row_begin, int row_count) {
    __shared__ float s_lo[kElemThreads / 32], s_hi[kElemThreads / 32];
    const int N = p.N;
    const size_t n = (size_t)N * N;
    const int k = *p.iter;
    const int slot = (k + 1) % p.D;
    for (int rr = blockIdx.x; rr < row_count; rr += gridDim.x) {
        const int R = row_begin + rr;  // global row: slice * N + i
        const int slice = R / N, i = R - slice * N;
        const int m = p.seg_of_row[i];
        const size_t ro = (size_t)i * N;
        const float* u = p.u + ((size_t)slice * p.M + m) * n + ro;
        const float* l = p.lam + ((size_t)slice * p.M + m) * n + ro;
        float* x = p.xseg + (size_t)slice * n + ro;
        float* xid = (p.need[m] & 1) ? p.hist + ((size_t)slot * 3 + DADMM_Q_NONE) * p.S * n + (size_t)slice * n + ro
                                     : nullptr;
        float lo = INFINITY, hi = -INFINITY;
        for (int j = threadIdx.x; j < N; j += kElemThreads) {
            const float v = fmaf(l[j], p.inv_rho, u[j]);  // u + lambda / rho
            float xv = x[j];
            for (int e = 0; e < p.E2; ++e) xv = fmaf(-p.eta2rho, xv - v, xv);
            x[j] = xv;
            if (xid) xid[j] = xv;
            lo = fminf(lo, xv);
            hi = fmaxf(hi, xv);
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
            for (int w = 1; w < kElemThreads / 32; ++w) {
                lo = fminf(lo, s_lo[w]);
                hi = fmaxf(hi, s_hi[w]);
            }
            atomicMin(p.lo_key + slice * p.M + m, float_key(lo));
            atomicMax(p.hi_key + slice * p.M + m, float_key(hi));
        }
        __syncthreads();
    }
}

// node m's view of row i at time k (= the current iteration kcur, or kcur + 1):
// the message version the relay rule gives, or, in lossy steps, the one held
__device__ __forceinline__ const float* view_row(const ElemParams& p, int slice, int m, int i, int k, int kcur) {
    const int seg = p.seg_of_row[i];
    const int mi = m * p.M + seg;
    const int j = p.held ? p.held[((size_t)(kcur - *p.k_first) * 2 + (k - kcur)) * p.M * p.M + mi] : k - p.lag[mi];
    if (j < 1) return nullptr;
    const size_t n = (size_t)p.N * p.N;
    return p.hist + (((size_t)(j % p.D) * 3 + p.kind[mi]) * p.S + slice) * n + (size_t)i * p.N;
}

// w = lambda - rho x, the part of the next Algorithm 2 step that stays fixed
// during its inner steps (the view x^{k+1} is the one that step reads)
__device__ __forceinline__ float4 wfix4(float4 l, float4 x, float rho) {
    return make_float4(fmaf(-rho, x.x, l.x), fmaf(-rho, x.y, l.y), fmaf(-rho, x.z, l.z), fmaf(-rho, x.w, l.w));
}

// Eq. 24 on every node: lambda_m <- lambda_m + rho (u_m - x_m^{k+1}), and
// w_m = lambda_m - rho x_m^{k+1} for the next iteration's Algorithm 2; FP64
// partial norms per block (gap2 over all nodes; change and norm of node 0's view)
__global__ void __launch_bounds__(kElemThreads) dual_kernel(const ElemParams p, int node_begin, int slice_begin) {
    __shared__ double s_red[3][kElemThreads / 32];
    const int N = p.N;
    const size_t n = (size_t)N * N;
    const int k = *p.iter;
    const int slice = slice_begin + blockIdx.y;
    const int node = node_begin + blockIdx.x / kDualPerNode;
    const int part = blockIdx.x % kDualPerNode;
    double gap = 0.0, chg = 0.0, nrm = 0.0;
    for (int i = part; i < N; i += kDualPerNode) {
        const size_t o = ((size_t)slice * p.M + node) * n + (size_t)i * N;
        const float* u = p.u + o;
        float* l = p.lam + o;
        float* wr = p.w + o;
        const float* x1 = view_row(p, slice, node, i, k + 1, k);
        const float* x0 = node == 0 ? view_row(p, slice, node, i, k, k) : nullptr;
        float g = 0.f, c = 0.f, q = 0.f;
        auto update = [&](float uv, float xv, float& lv, float xo) {
            const float pr = uv - xv;
            g = fmaf(pr, pr, g);
            lv = fmaf(p.rho, pr, lv);
            if (node == 0) {
                c = fmaf(xv - xo, xv - xo, c);
                q = fmaf(xo, xo, q);
            }
        };
        if ((N & 3) == 0) {
            // rows are 16-byte aligned: two float4 of u, x and lambda per thread are
            // loaded before any store, so the loads of a row are in flight together;
            // the node's own u, lambda and w pass through L2 once (evict-first, .cs),
            // the views of x are shared by the nodes and keep normal priority
            const int N4 = N >> 2;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int j = threadIdx.x; j < N4; j += 2 * kElemThreads) {
                const int jb = j + kElemThreads;
                const bool two = jb < N4;
                const float4 ua = __ldcs(reinterpret_cast<const float4*>(u) + j);
                const float4 ub = two ? __ldcs(reinterpret_cast<const float4*>(u) + jb) : z4;
                const float4 xa = x1 ? __ldg(reinterpret_cast<const float4*>(x1) + j) : z4;
                const float4 xb = (x1 && two) ? __ldg(reinterpret_cast<const float4*>(x1) + jb) : z4;
                float4 la = __ldcs(reinterpret_cast<const float4*>(l) + j);
                float4 lb = two ? __ldcs(reinterpret_cast<const float4*>(l) + jb) : z4;
                float4 oa = z4, ob = z4;
                if (node == 0 && x0) {
                    oa = __ldg(reinterpret_cast<const float4*>(x0) + j);
                    if (two) ob = __ldg(reinterpret_cast<const float4*>(x0) + jb);
                }
                update(ua.x, xa.x, la.x, oa.x);
                update(ua.y, xa.y, la.y, oa.y);
                update(ua.z, xa.z, la.z, oa.z);
                update(ua.w, xa.w, la.w, oa.w);
                __stcs(reinterpret_cast<float4*>(l) + j, la);
                __stcs(reinterpret_cast<float4*>(wr) + j, wfix4(la, xa, p.rho));
                if (two) {
                    update(ub.x, xb.x, lb.x, ob.x);
                    update(ub.y, xb.y, lb.y, ob.y);
                    update(ub.z, xb.z, lb.z, ob.z);
                    update(ub.w, xb.w, lb.w, ob.w);
                    __stcs(reinterpret_cast<float4*>(l) + jb, lb);
                    __stcs(reinterpret_cast<float4*>(wr) + jb, wfix4(lb, xb, p.rho));
                }
            }
        } else {
            for (int j = threadIdx.x; j < N; j += kElemThreads) {
                float lv = l[j];
                const float xv = x1 ? x1[j] : 0.f;
                update(u[j], xv, lv, x0 ? x0[j] : 0.f);
                l[j] = lv;
                wr[j] = fmaf(-p.rho, xv, lv);
            }
        }
        gap += g;
        chg += c;
        nrm += q;
    }
    for (int o = 16; o > 0; o >>= 1) {
        gap += __shfl_xor_sync(0xffffffffu, gap, o);
        chg += __shfl_xor_sync(0xffffffffu, chg, o);
        nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_red[0][w] = gap;
        s_red[1][w] = chg;
        s_red[2][w] = nrm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int v = 0; v < kElemThreads / 32; ++v) {
            a += s_red[0][v];
            b += s_red[1][v];
            c += s_red[2][v];
        }
        double* d = p.dual_part + (((size_t)slice * p.M + node) * kDualPerNode + part) * 3;
        d[0] = a;
        d[1] = b;
        d[2] = c;
    }
}

// sum of squared residuals (last inner step) per slice
// sum of squares of the residual lines; line a is stored as h_a r_a and
// mx[a] = 1 / h_a = max(|cos|, |sin|) restores r_a
__global__ void __launch_bounds__(kElemThreads) resid_kernel(const float* resid, const float* mx, int A, int B,
                                                             double* part) {
    __shared__ double s_red[kElemThreads / 32];
    const int slice = blockIdx.y;
    double acc = 0.0;
    for (int a = blockIdx.x; a < A; a += kResPerSlice) {
        const float* r = resid + ((size_t)slice * A + a) * B;
        const float m = mx[a];
        float t = 0.f;
        for (int b = threadIdx.x; b < B; b += kElemThreads) {
            const float v = r[b] * m;
            t = fmaf(v, v, t);
        }
        acc += t;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kElemThreads / 32; ++w) t += s_red[w];
        part[(size_t)slice * kResPerSlice + blockIdx.x] = t;
    }
}

struct FinParams {
    const double* dual_part;
    const double* res_part;
    const long long* nnz;      // [S][M] entropy-coded JPEG message bytes
    const int32_t* recv;       // [M][3]
    const int32_t* seg_rows;   // [M]
    double* stats;             // [kStatsCap][S][DADMM_NSTAT]
    int32_t* iter;
    int* status;
    int S, M, N, km_k;
};

// deterministic reduction of the partials, message bytes, counter increment
__global__ void finalize_kernel(const FinParams p) {
    __shared__ double s[4][256];
    const int k = *p.iter;
    for (int slice = 0; slice < p.S; ++slice) {
        double a = 0.0, b = 0.0, c = 0.0, r = 0.0, by = 0.0;
        const int nparts = p.M * kDualPerNode;
        for (int q = threadIdx.x; q < nparts; q += blockDim.x) {
            const double* d = p.dual_part + ((size_t)slice * nparts + q) * 3;
            a += d[0];
            b += d[1];
            c += d[2];
        }
        for (int q = threadIdx.x; q < kResPerSlice; q += blockDim.x) r += p.res_part[(size_t)slice * kResPerSlice + q];
        int bits = 0;
        while ((1 << bits) < p.km_k) ++bits;
        for (int m = threadIdx.x; m < p.M; m += blockDim.x) {
            const double len = (double)p.seg_rows[m] * p.N;
            by += p.recv[m * 3 + 0] * 4.0 * len;
            by += p.recv[m * 3 + 1] * (bits * len / 8.0 + 4.0 * p.km_k);
            by += p.recv[m * 3 + 2] * ((double)p.nnz[slice * p.M + m] + 8.0);  // entropy-coded blocks + (lo, hi)
        }
        s[0][threadIdx.x] = a;
        s[1][threadIdx.x] = b;
        s[2][threadIdx.x] = c;
        s[3][threadIdx.x] = r;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w)
                for (int t = 0; t < 4; ++t) s[t][threadIdx.x] += s[t][threadIdx.x + w];
            __syncthreads();
        }
        // bytes: exact integers in double, any order
        for (int o = 16; o > 0; o >>= 1) by += __shfl_xor_sync(0xffffffffu, by, o);
        __shared__ double s_by[8];
        if ((threadIdx.x & 31) == 0) s_by[threadIdx.x >> 5] = by;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tb = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tb += s_by[w];
            double* st = p.stats + ((size_t)(k % kStatsCap) * p.S + slice) * DADMM_NSTAT;
            st[0] = s[0][0];
            st[1] = s[1][0];
            st[2] = s[2][0];
            st[3] = s[3][0];
            st[4] = tb;
            for (int t = 0; t < 4; ++t)
                if (!isfinite(s[t][0])) atomicOr(p.status, 2);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *p.iter = k + 1;
}

__global__ void home_view_kernel(const float* hist, const int32_t* iter, const int32_t* seg_of_row,
                                 const int32_t* home, float* out, int N, int S, int D) {
    const size_t n = (size_t)N * N;
    const int k = *iter;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)S * n;
         e += (size_t)gridDim.x * blockDim.x) {
        const int slice = (int)(e / n);
        const size_t o = e - (size_t)slice * n;
        const int i = (int)(o / N);
        if (k < 1) {
            out[e] = 0.f;
            continue;
        }
        const int m = seg_of_row[i];
        out[e] = hist[(((size_t)(k % D) * 3 + home[m]) * S + slice) * n + o];
    }
}

// ------------------------------------------------------------------
// neighbour-averaged consensus variant (the decentralized analogue of the
// standard ADMM x-update, Eq. 9): every node keeps its own x_m [S][M][N][N]
// (in the state's x array) and averages the full-image messages of its closed
// neighbourhood; the message planes are [3][S][M][N][N] (in the history array)
// ------------------------------------------------------------------
struct ConsParams {
    ElemParams e;
    float* x;              // [S][M][N][N] every node's consensus image
    float* msg;            // [3][S][M][N][N] dequantized messages (plane 0: identity)
    const int32_t* nb_ptr; // [M+1] closed neighbourhood of each node
    const int32_t* nb;     // sender j | quantizer << 16: the node itself first, then its neighbours
};

// v_j = u_j + lambda_j / rho: node j's message before quantization (identity
// plane and codec source), and its min / max for the JPEG sample map
__global__ void __launch_bounds__(kElemThreads) cons_message_kernel(const ConsParams c, int row_begin, int row_count) {
    __shared__ float s_lo[kElemThreads / 32], s_hi[kElemThreads / 32];
    const ElemParams& p = c.e;
    const int N = p.N;
    for (int rr = blockIdx.x; rr < row_count; rr += gridDim.x) {
        const int R = row_begin + rr;  // (slice * M + j) * N + i
        const int img = R / N;         // slice * M + j
        const size_t o = (size_t)R * N;
        float lo = INFINITY, hi = -INFINITY;
        for (int j = threadIdx.x; j < N; j += kElemThreads) {
            const float v = fmaf(p.lam[o + j], p.inv_rho, p.u[o + j]);
            c.msg[o + j] = v;
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
        for (int q = 16; q > 0; q >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, q));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, q));
        }
        if ((threadIdx.x & 31) == 0) {
            s_lo[threadIdx.x >> 5] = lo;
            s_hi[threadIdx.x >> 5] = hi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kElemThreads / 32; ++w) {
                lo = fminf(lo, s_lo[w]);
                hi = fmaxf(hi, s_hi[w]);
            }
            atomicMin(p.lo_key + img, float_key(lo));
            atomicMax(p.hi_key + img, float_key(hi));
        }
        __syncthreads();
    }
}

// x_m^{k+1} = mean over the closed neighbourhood of the received messages;
// lambda_m += rho (u_m - x_m^{k+1}), w_m = lambda_m - rho x_m^{k+1}; FP64
// partial norms as dual_kernel (the change and norm statistics of node 0's x)
__global__ void __launch_bounds__(kElemThreads) cons_dual_kernel(const ConsParams c, int node_begin, int slice_begin) {
    __shared__ double s_red[3][kElemThreads / 32];
    const ElemParams& p = c.e;
    const int N = p.N, M = p.M;
    const size_t n = (size_t)N * N, plane = (size_t)p.S * M * n;
    const int slice = slice_begin + blockIdx.y;
    const int node = node_begin + blockIdx.x / kDualPerNode;
    const int part = blockIdx.x % kDualPerNode;
    const int e0 = c.nb_ptr[node], e1 = c.nb_ptr[node + 1];
    const float inv_cnt = 1.0f / (float)(e1 - e0);
    double gap = 0.0, chg = 0.0, nrm = 0.0;
    for (int i = part; i < N; i += kDualPerNode) {
        const size_t o = ((size_t)slice * M + node) * n + (size_t)i * N;
        float g = 0.f, ch = 0.f, q = 0.f;
        for (int j = threadIdx.x; j < N; j += kElemThreads) {
            float acc = 0.f;
            for (int e = e0; e < e1; ++e) {
                const int src = c.nb[e] & 0xFFFF, kd = c.nb[e] >> 16;
                acc += c.msg[(size_t)kd * plane + ((size_t)slice * M + src) * n + (size_t)i * N + j];
            }
            const float xn = acc * inv_cnt;
            if (node == 0) {
                const float xo = c.x[o + j];
                ch = fmaf(xn - xo, xn - xo, ch);
                q = fmaf(xo, xo, q);
            }
            c.x[o + j] = xn;
            const float pr = p.u[o + j] - xn;
            g = fmaf(pr, pr, g);
            const float ln = fmaf(p.rho, pr, p.lam[o + j]);
            p.lam[o + j] = ln;
            p.w[o + j] = fmaf(-p.rho, xn, ln);
        }
        gap += g;
        chg += ch;
        nrm += q;
    }
    for (int q = 16; q > 0; q >>= 1) {
        gap += __shfl_xor_sync(0xffffffffu, gap, q);
        chg += __shfl_xor_sync(0xffffffffu, chg, q);
        nrm += __shfl_xor_sync(0xffffffffu, nrm, q);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_red[0][w] = gap;
        s_red[1][w] = chg;
        s_red[2][w] = nrm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, cc = 0.0;
        for (int v = 0; v < kElemThreads / 32; ++v) {
            a += s_red[0][v];
            b += s_red[1][v];
            cc += s_red[2][v];
        }
        double* d = p.dual_part + (((size_t)slice * M + node) * kDualPerNode + part) * 3;
        d[0] = a;
        d[1] = b;
        d[2] = cc;
    }
}

// w_m = lambda_m^k - rho x_m^k from the state as it is (after the state was
// initialised or written from outside): x_m^k is the node's view of the
// current iteration (segments variant, the relay or held version) or its own x
// (consensus variant, xnode non-null)
__global__ void __launch_bounds__(kElemThreads) wprep_kernel(const ElemParams p, const float* xnode) {
    const int N = p.N;
    const size_t n = (size_t)N * N;
    const int k = *p.iter;
    const long long rows = (long long)p.S * p.M * N;
    for (long long R = blockIdx.x; R < rows; R += gridDim.x) {  // (slice * M + m) * N + i
        const int img = (int)(R / N), i = (int)(R - (long long)img * N);
        const int slice = img / p.M, m = img - slice * p.M;
        const size_t o = (size_t)R * N;
        const float* xr = xnode ? xnode + o : view_row(p, slice, m, i, k, k);
        for (int j = threadIdx.x; j < N; j += kElemThreads)
            p.w[o + j] = fmaf(-p.rho, xr ? xr[j] : 0.f, p.lam[o + j]);
    }
}

// the consensus reconstruction: the mean of the nodes' x
__global__ void cons_view_kernel(const float* x, float* out, int N, int S, int M) {
    const size_t n = (size_t)N * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)S * n;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t slice = e / n, o = e - slice * n;
        float acc = 0.f;
        for (int m = 0; m < M; ++m) acc += x[(slice * M + m) * n + o];
        out[e] = acc / (float)M;
    }
}

// ------------------------------------------------------------------
// elementwise building blocks (linear combinations, FP64 dots)
// ------------------------------------------------------------------
struct LinComb {
    const float* x[4];
    float c[4];
};

template <int K>
__global__ void lincomb_kernel(const LinComb a, float* out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v = a.c[0] * a.x[0][i];
#pragma unroll
        for (int j = 1; j < K; ++j) v = fmaf(a.c[j], a.x[j][i], v);
        out[i] = v;
    }
}

constexpr int kDotBlocks = TOMO_DOT_SCRATCH - 1;

__global__ void dot_partial_kernel(const float* x, const float* y, long long n, double* part) {
    __shared__ double s[kElemThreads / 32];
    double acc = 0.0;
    for (long long base = (long long)blockIdx.x * kElemThreads; base < n; base += (long long)kDotBlocks * kElemThreads) {
        const long long i = base + threadIdx.x;
        if (i < n) acc = fma((double)x[i], (double)y[i], acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kElemThreads / 32; ++w) t += s[w];
        part[blockIdx.x] = t;
    }
}

__global__ void dot_final_kernel(const double* part, double* out) {
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < kDotBlocks; ++b) t += part[b];
        *out = t;
    }
}

// ------------------------------------------------------------------
// host
// ------------------------------------------------------------------
static void relay_tables(int M, const std::vector<int32_t>& adj, std::vector<int>& dist,
                         std::vector<int>& first) {
    dist.assign((size_t)M * M, -1);
    first.assign((size_t)M * M, -1);
    for (int s = 0; s < M; ++s) {
        int* d = &dist[(size_t)s * M];
        std::queue<int> q;
        d[s] = 0;
        q.push(s);
        while (!q.empty()) {
            const int x = q.front();
            q.pop();
            for (int y = 0; y < M; ++y)
                if (adj[(size_t)x * M + y] && d[y] < 0) {
                    d[y] = d[x] + 1;
                    q.push(y);
                }
        }
        for (int m = 0; m < M; ++m) {
            if (m == s) {
                first[(size_t)s * M + m] = s;
                continue;
            }
            if (d[m] < 0) continue;
            int cur = m;
            while (d[cur] > 1) {  // lowest-id neighbour one hop closer to s
                int par = -1;
                for (int pp = 0; pp < M && par < 0; ++pp)
                    if (adj[(size_t)pp * M + cur] && d[pp] == d[cur] - 1) par = pp;
                cur = par;
            }
            first[(size_t)s * M + m] = cur;
        }
    }
}

static void free_dadmm(Dadmm* h) {
    if (!h) return;
    h->drop_graphs();
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->own) cudaStreamDestroy(h->own);
    for (cudaEvent_t e : h->pev) cudaEventDestroy(e);
    void* ptrs[] = {h->d_angs, h->d_bk, h->d_pitems, h->d_bitems, h->d_pplain, h->d_bplain, h->d_lag, h->d_kind,
                    h->d_seg_of_row, h->d_need, h->d_recv, h->d_home, h->d_eta1, h->d_mx, h->d_km, h->d_jp,
                    h->d_nb_ptr, h->d_nb, h->d_eta0};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete h;
}

// the projector and backprojector work lists of the handle's launch shapes, in
// the plain (per slice and node) and batched forms; replaces earlier lists
static void build_lists(Dadmm& h) {
    const int M = h.M, S = h.S, A = h.A;
    std::vector<ProjItem> pplain;
    std::vector<BpItem> bplain;
    h.p_range.assign((size_t)2 * S * M, 0);
    h.b_range.assign((size_t)2 * S * M, 0);
    for (int sl = 0; sl < S; ++sl)
        for (int m = 0; m < M; ++m) {
            const int a0 = h.node_ang_ptr[m], na = h.node_ang_ptr[m + 1] - a0;
            const int sn = sl * M + m;
            h.p_range[2 * sn] = (int)pplain.size();
            if (na > 0 && sl % h.proj_slices == 0)  // slice groups: the first slice's items cover the group
                build_proj_items(*h.g, h.angs, a0, na, sn, sl * A, pplain, h.proj_bins4);
            h.p_range[2 * sn + 1] = (int)pplain.size();
            h.b_range[2 * sn] = (int)bplain.size();
            if (na > 0) build_bp_items(*h.g, a0, na, sn, sl * A, m, sl, bplain, h.bp_tile_x);
            h.b_range[2 * sn + 1] = (int)bplain.size();
        }
    // nodes without angles still need the u-step (pure proximal term)
    for (int sl = 0; sl < S; ++sl)
        for (int m = 0; m < M; ++m) {
            const int sn = sl * M + m;
            if (h.b_range[2 * sn] == h.b_range[2 * sn + 1]) {
                build_bp_items(*h.g, h.node_ang_ptr[m], 0, sn, sl * A, m, sl, bplain, h.bp_tile_x);
                h.b_range[2 * sn + 1] = (int)bplain.size();
            }
        }
    // batched order: node-major, as the plain lists, so that the blocks in flight
    // work on few nodes at a time and each node's image stays in L2; with slice
    // pairs, the items of the even slices, each also covering the next slice
    std::vector<BpItem> bbatch;
    if (h.bp_slices == 2) {
        for (const BpItem& it : bplain)
            if (it.slice % 2 == 0) bbatch.push_back(it);
    } else {
        bbatch = bplain;
    }
    for (void* q : {(void*)h.d_pitems, (void*)h.d_bitems, (void*)h.d_pplain, (void*)h.d_bplain})
        if (q) cudaFree(q);
    h.d_pitems = h.d_pplain = nullptr;
    h.d_bitems = h.d_bplain = nullptr;
    h.d_pitems = device_upload(pplain);
    h.d_bitems = device_upload(bbatch);
    h.d_pplain = device_upload(pplain);
    h.d_bplain = device_upload(bplain);
    h.n_pitems = (int)pplain.size();
    h.n_bitems = (int)bbatch.size();
    h.grid_proj = persistent_grid_project(h.proj_slices);
    h.grid_bp = persistent_grid_backproject(true, h.bp_tile_x, h.bp_slices);
    h.drop_graphs();
}

struct WsPtrs {
    float* uT;
    float* w;            // [S][M][N][N] lambda_m - rho x_m (the fixed part of the Algorithm 2 step)
    float* resid;
    int* counters;
    unsigned* lo;
    unsigned* hi;
    long long* nnz;      // [S][M] entropy-coded JPEG message bytes
    int32_t* held;       // lossy steps: k_first, then the held-version table
    int16_t* coefs;      // quantized blocks of the JPEG segments
    uint32_t* bits;      // their entropy-coding bit buffers
    double* dual;
    double* res;
    double* stats;
    int* status;
};

static WsPtrs ws_ptrs(const Dadmm& h, void* ws) {
    char* b = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    WsPtrs w;
    w.uT = (float*)(b + h.off_uT);
    w.w = (float*)(b + h.off_w);
    w.resid = (float*)(b + h.off_resid);
    w.counters = (int*)(b + h.off_counters);
    w.lo = (unsigned*)(b + h.off_lo);
    w.hi = (unsigned*)(b + h.off_hi);
    w.nnz = (long long*)(b + h.off_nnz);
    w.held = h.max_stale > 0 ? (int32_t*)(b + h.off_held) : nullptr;
    w.coefs = (int16_t*)(b + h.off_coefs);
    w.bits = (uint32_t*)(b + h.off_bits);
    w.dual = (double*)(b + h.off_dual);
    w.res = (double*)(b + h.off_res);
    w.stats = (double*)(b + h.off_stats);
    w.status = (int*)(b + h.off_status);
    return w;
}

static ElemParams elem_params(const Dadmm& h, const dadmm_state& st, const WsPtrs& w) {
    ElemParams p{};
    p.u = st.u;
    p.lam = st.lam;
    p.xseg = st.xseg;
    p.hist = st.hist;
    p.iter = st.iter;
    p.seg_of_row = h.d_seg_of_row;
    p.lag = h.d_lag;
    p.kind = h.d_kind;
    p.held = h.lossy ? w.held + 4 : nullptr;  // the first 16 bytes hold k_first
    p.k_first = h.lossy ? w.held : nullptr;
    p.need = h.d_need;
    p.lo_key = w.lo;
    p.hi_key = w.hi;
    p.dual_part = w.dual;
    p.w = w.w;
    p.N = h.N;
    p.S = h.S;
    p.M = h.M;
    p.D = h.D;
    p.E2 = h.E2;
    p.rho = (float)h.rho;
    p.eta2rho = (float)(h.eta2 * h.rho);
    p.inv_rho = (float)(1.0 / h.rho);
    return p;
}

// projector launch parameters of the iteration: u -> h_a (h_a P u - d) in the
// residual buffer (work list, queue counter and item count set by the caller)
static ProjParams proj_params(const Dadmm& h, const dadmm_state& st, const float* sino, const WsPtrs& w) {
    ProjParams pp{};
    if (h.has_maps) {
        pp.map = h.map_u;
        pp.mapT = h.map_uT;
        pp.has_map = pp.has_mapT = 1;
    }
    pp.img = st.u;
    pp.out = w.resid;
    pp.sub = sino;
    pp.angs = h.d_angs;
    pp.status = w.status;
    pp.N = h.N;
    pp.B = h.B;
    pp.ptab = h.g->d_ptab;
    pp.prescale = 1;  // the residual is stored as h_a r_a, the form the backprojector stages
    pp.map_rows = h.map_rows;
    pp.pair_img = h.M;   // slice-pair items: the next slice's image of the node
    pp.pair_rows = h.A;  // ... and its residual lines
    return pp;
}

// backprojector (u-step) launch parameters of the iteration
static BpParams bp_params(const Dadmm& h, const dadmm_state& st, const WsPtrs& w) {
    BpParams bp{};
    bp.sino = w.resid;
    bp.bk = h.d_bk;
    bp.status = w.status;
    bp.N = h.N;
    bp.B = h.B;
    bp.prescaled = 1;
    bp.pair_img = h.M;  // slice-pair items: the next slice's image of the node
    bp.pair_rows = h.A;  // ... and its residual lines
    bp.view.eta1 = h.d_eta1;
    bp.view.u = st.u;
    bp.view.uT = h.has_maps ? w.uT : nullptr;
    bp.view.w = w.w;
    bp.view.rho = (float)h.rho;
    return bp;
}

// enqueue one full iteration on stream st
static void enqueue_iteration(Dadmm& h, const dadmm_state& st, const float* sino, const WsPtrs& w,
                              cudaStream_t s) {
    const bool batched = h.mode == DADMM_MODE_BATCHED;
    int phase = 0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    TOMO_CUDA(cudaStreamIsCapturing(s, &cap));
    auto mark = [&]() {  // boundary before phase `phase`; a graph node when capturing
        if (h.profiling)
            TOMO_CUDA(cudaEventRecordWithFlags(h.pev[phase], s,
                                               cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0));
        ++phase;
    };
    const size_t SM = (size_t)h.S * h.M;
    // per-iteration resets: work queues, segment min/max keys, JPEG counters
    TOMO_CUDA(cudaMemsetAsync(w.counters, 0, sizeof(int) * (2 * h.E1 + 2), s));
    TOMO_CUDA(cudaMemsetAsync(w.lo, 0xFF, sizeof(unsigned) * SM, s));
    TOMO_CUDA(cudaMemsetAsync(w.hi, 0x00, sizeof(unsigned) * SM, s));
    TOMO_CUDA(cudaMemsetAsync(w.nnz, 0, sizeof(long long) * SM, s));

    ProjParams pp = proj_params(h, st, sino, w);
    BpParams bp = bp_params(h, st, w);

    for (int e = 0; e < h.E1; ++e) {
        if (batched) {
            mark();
            pp.items = h.d_pitems;
            pp.n_items = h.n_pitems;
            pp.counter = w.counters + 2 * e;
            launch_project(pp, std::min(h.grid_proj, h.n_pitems), s, h.proj_slices);
            mark();
            bp.items = h.d_bitems;
            bp.n_items = h.n_bitems;
            bp.counter = w.counters + 2 * e + 1;
            launch_backproject_ustep(bp, std::min(h.grid_bp, h.n_bitems), s, h.bp_tile_x, h.bp_slices);
        } else {
            mark();
            for (int sn = 0; sn < h.S * h.M; ++sn) {
                pp.items = h.d_pplain + h.p_range[2 * sn];
                pp.n_items = h.p_range[2 * sn + 1] - h.p_range[2 * sn];
                pp.counter = nullptr;
                launch_project(pp, pp.n_items, s, h.proj_slices);
            }
            mark();
            for (int sn = 0; sn < h.S * h.M; ++sn) {
                bp.items = h.d_bplain + h.b_range[2 * sn];
                bp.n_items = h.b_range[2 * sn + 1] - h.b_range[2 * sn];
                bp.counter = nullptr;
                launch_backproject_ustep(bp, bp.n_items, s, h.bp_tile_x);
            }
        }
    }

    ElemParams ep = elem_params(h, st, w);
    DadmmCodec cp{};
    cp.xseg = st.xseg;
    cp.hist = st.hist;
    cp.iter = st.iter;
    cp.N = h.N;
    cp.S = h.S;
    cp.D = h.D;
    cp.seed = h.seed;
    cp.lo_key = w.lo;
    cp.hi_key = w.hi;
    cp.coefs = w.coefs;
    cp.bits = w.bits;
    cp.jbytes = w.nnz;
    cp.M = h.M;
    const size_t nn = (size_t)h.N * h.N;
    if (h.variant == DADMM_VARIANT_CONSENSUS) {
        // messages: full images of every node, one exchange (no ring)
        ConsParams cs{};
        cs.e = ep;
        cs.x = st.xseg;
        cs.msg = st.hist;
        cs.nb_ptr = h.d_nb_ptr;
        cs.nb = h.d_nb;
        cp.xseg = st.hist;  // the codecs read the identity plane
        cp.plane_stride = (size_t)h.S * h.M * nn;
        cp.slot_stride = 0;
        const int rows = h.S * h.M * h.N;
        if (batched) {
            mark();
            cons_message_kernel<<<std::min(rows, 152 * 8), kElemThreads, 0, s>>>(cs, 0, rows);
            TOMO_CUDA(cudaGetLastError());
            mark();
            cp.tasks = h.d_km;
            launch_kmeans_dadmm(cp, h.km_k, h.km_iters, 0, h.n_km, s);
            mark();
            cp.tasks = h.d_jp;
            launch_jpeg_dadmm(cp, h.jpeg_q, h.max_jp_rows, 0, h.n_jp, s);
            launch_jpeg_entropy_dadmm(cp, 0, h.n_jp, s);
            mark();
            cons_dual_kernel<<<dim3(h.M * kDualPerNode, h.S), kElemThreads, 0, s>>>(cs, 0, 0);
            TOMO_CUDA(cudaGetLastError());
        } else {
            mark();
            for (int img = 0; img < h.S * h.M; ++img) {
                cons_message_kernel<<<h.N, kElemThreads, 0, s>>>(cs, img * h.N, h.N);
                TOMO_CUDA(cudaGetLastError());
            }
            mark();
            cp.tasks = h.d_km;
            for (int t = 0; t < h.n_km; ++t) launch_kmeans_dadmm(cp, h.km_k, h.km_iters, t, 1, s);
            mark();
            cp.tasks = h.d_jp;
            for (int t = 0; t < h.n_jp; ++t) {
                launch_jpeg_dadmm(cp, h.jpeg_q, h.N, t, 1, s);
                launch_jpeg_entropy_dadmm(cp, t, 1, s);
            }
            mark();
            for (int sl = 0; sl < h.S; ++sl)
                for (int m = 0; m < h.M; ++m) {
                    cons_dual_kernel<<<dim3(kDualPerNode, 1), kElemThreads, 0, s>>>(cs, m, sl);
                    TOMO_CUDA(cudaGetLastError());
                }
        }
    } else if (batched) {
        cp.plane_stride = (size_t)h.S * nn;
        cp.slot_stride = 3 * (size_t)h.S * nn;
        const int rows = h.S * h.N;
        mark();
        xstep_kernel<<<std::min(rows, 152 * 8), kElemThreads, 0, s>>>(ep, 0, rows);
        TOMO_CUDA(cudaGetLastError());
        mark();
        cp.tasks = h.d_km;
        launch_kmeans_dadmm(cp, h.km_k, h.km_iters, 0, h.n_km, s);
        mark();
        cp.tasks = h.d_jp;
        launch_jpeg_dadmm(cp, h.jpeg_q, h.max_jp_rows, 0, h.n_jp, s);
        launch_jpeg_entropy_dadmm(cp, 0, h.n_jp, s);
        mark();
        dual_kernel<<<dim3(h.M * kDualPerNode, h.S), kElemThreads, 0, s>>>(ep, 0, 0);
        TOMO_CUDA(cudaGetLastError());
    } else {
        cp.plane_stride = (size_t)h.S * nn;
        cp.slot_stride = 3 * (size_t)h.S * nn;
        mark();
        for (int sl = 0; sl < h.S; ++sl)
            for (int m = 0; m < h.M; ++m) {
                const int r0 = h.seg_row_ptr[m], r1 = h.seg_row_ptr[m + 1];
                xstep_kernel<<<r1 - r0, kElemThreads, 0, s>>>(ep, sl * h.N + r0, r1 - r0);
                TOMO_CUDA(cudaGetLastError());
            }
        mark();
        cp.tasks = h.d_km;
        for (int sl = 0; sl < h.S; ++sl)
            for (int m = 0; m < h.M; ++m) {
                const int ki = h.km_index[sl * h.M + m];
                if (ki >= 0) launch_kmeans_dadmm(cp, h.km_k, h.km_iters, ki, 1, s);
            }
        mark();
        cp.tasks = h.d_jp;
        for (int sl = 0; sl < h.S; ++sl)
            for (int m = 0; m < h.M; ++m) {
                const int ji = h.jp_index[sl * h.M + m];
                if (ji >= 0) {
                    launch_jpeg_dadmm(cp, h.jpeg_q, h.seg_row_ptr[m + 1] - h.seg_row_ptr[m], ji, 1, s);
                    launch_jpeg_entropy_dadmm(cp, ji, 1, s);
                }
            }
        mark();
        for (int sl = 0; sl < h.S; ++sl)
            for (int m = 0; m < h.M; ++m) {
                dual_kernel<<<dim3(kDualPerNode, 1), kElemThreads, 0, s>>>(ep, m, sl);
                TOMO_CUDA(cudaGetLastError());
            }
    }
    mark();
    resid_kernel<<<dim3(kResPerSlice, h.S), kElemThreads, 0, s>>>(w.resid, h.d_mx, h.A, h.B, w.res);
    TOMO_CUDA(cudaGetLastError());
    FinParams fp{};
    fp.dual_part = w.dual;
    fp.res_part = w.res;
    fp.nnz = w.nnz;
    fp.recv = h.d_recv;
    fp.seg_rows = h.d_need + h.M;  // second half of the need table holds the segment row counts
    fp.stats = w.stats;
    fp.iter = st.iter;
    fp.status = w.status;
    fp.S = h.S;
    fp.M = h.M;
    fp.N = h.N;
    fp.km_k = h.km_k;
    finalize_kernel<<<1, 256, 0, s>>>(fp);
    TOMO_CUDA(cudaGetLastError());
    mark();  // end of the last phase
}

// values of the state's x and history arrays (segment variant: x~ [S][N][N] and the
// message ring [D][3][S][N][N]; consensus: x [S][M][N][N] and messages [3][S][M][N][N])
static size_t x_values(const Dadmm& h) {
    const size_t n = (size_t)h.N * h.N;
    return h.variant == DADMM_VARIANT_CONSENSUS ? (size_t)h.S * h.M * n : (size_t)h.S * n;
}
static size_t hist_values(const Dadmm& h) {
    const size_t n = (size_t)h.N * h.N;
    return h.variant == DADMM_VARIANT_CONSENSUS ? 3 * (size_t)h.S * h.M * n : (size_t)h.D * 3 * h.S * n;
}

// device status word of a dADMM workspace: bit 0 projector extent (internal
// error), bit 1 non-finite statistics, bit 2 a bounded wait gave up
static void check_status_word(int status, tomo_status* numeric) {
    if (status & 4) fail(TOMO_ERR_TIMEOUT, "a bounded wait for a staged image band gave up; the iterate is incomplete");
    if (status & 1) fail(TOMO_ERR_CUDA, "projector staging extent exceeded (internal error)");
    if (status & 2) *numeric = TOMO_ERR_NUMERIC;
}

}  // namespace tomo

using namespace tomo;

extern "C" {

tomo_status tomo_lincomb(int64_t n, int k, const float* const* x, const float* coef, float* out,
                         tomo_stream_t stream) {
    return guard([&] {
        TOMO_REQUIRE(n >= 0 && k >= 1 && k <= 4 && x && coef && out, "bad tomo_lincomb arguments");
        LinComb a{};
        for (int j = 0; j < k; ++j) {
            TOMO_REQUIRE(x[j] != nullptr, "tomo_lincomb: NULL input");
            a.x[j] = x[j];
            a.c[j] = coef[j];
        }
        if (n == 0) return;
        const int grid = (int)std::min<long long>((n + kElemThreads - 1) / kElemThreads, 152LL * 16);
        cudaStream_t s = (cudaStream_t)stream;
        switch (k) {
            case 1: lincomb_kernel<1><<<grid, kElemThreads, 0, s>>>(a, out, n); break;
            case 2: lincomb_kernel<2><<<grid, kElemThreads, 0, s>>>(a, out, n); break;
            case 3: lincomb_kernel<3><<<grid, kElemThreads, 0, s>>>(a, out, n); break;
            default: lincomb_kernel<4><<<grid, kElemThreads, 0, s>>>(a, out, n); break;
        }
        TOMO_CUDA(cudaGetLastError());
    });
}

tomo_status tomo_dot(int64_t n, const float* x, const float* y, double* out, tomo_stream_t stream) {
    return guard([&] {
        TOMO_REQUIRE(n >= 0 && x && y && out, "bad tomo_dot arguments");
        cudaStream_t s = (cudaStream_t)stream;
        dot_partial_kernel<<<kDotBlocks, kElemThreads, 0, s>>>(x, y, n, out + 1);
        dot_final_kernel<<<1, 32, 0, s>>>(out + 1, out);
        TOMO_CUDA(cudaGetLastError());
    });
}

tomo_status dadmm_create(tomo_geometry_t gh, const dadmm_config* cfg, dadmm_t* out) {
    return guard([&] {
        TOMO_REQUIRE(out != nullptr && cfg != nullptr, "cfg and out must be non-NULL");
        *out = nullptr;
        Geometry* g = as_geometry(gh);
        check_device(*g);
        const dadmm_config& c = *cfg;
        TOMO_REQUIRE(c.N == g->N && c.n_bins == g->B && c.n_angles == g->A,
                     "config sizes differ from the geometry");
        TOMO_REQUIRE(c.S >= 1 && c.M >= 1 && c.M <= 127, "need S >= 1 and 1 <= M <= 127");
        TOMO_REQUIRE(c.node_ang_ptr && c.node_ang && c.seg_row_ptr && c.adj && c.edge_q && c.home_q && c.eta1,
                     "config arrays must be non-NULL");
        TOMO_REQUIRE(c.E1 >= 0 && c.E1 <= 1000 && c.E2 >= 0 && c.E2 <= 100000, "E1/E2 out of range");
        TOMO_REQUIRE(c.rho > 0.0 && std::isfinite(c.rho), "rho must be positive");
        TOMO_REQUIRE(c.mode == DADMM_MODE_BATCHED || c.mode == DADMM_MODE_PLAIN, "unknown mode");
        TOMO_REQUIRE(c.variant == DADMM_VARIANT_SEGMENTS || c.variant == DADMM_VARIANT_CONSENSUS, "unknown variant");
        const bool cons = c.variant == DADMM_VARIANT_CONSENSUS;
        TOMO_REQUIRE(!cons || c.max_stale == 0, "lost messages are a segment-variant feature");
        const int M = c.M, N = c.N, A = c.n_angles;
        // angle partition
        TOMO_REQUIRE(c.node_ang_ptr[0] == 0 && c.node_ang_ptr[M] == A, "node_ang_ptr must span all angles");
        std::vector<int> seen(A, 0);
        for (int m = 0; m < M; ++m) {
            TOMO_REQUIRE(c.node_ang_ptr[m + 1] >= c.node_ang_ptr[m], "node_ang_ptr must be non-decreasing");
            for (int q = c.node_ang_ptr[m]; q < c.node_ang_ptr[m + 1]; ++q) {
                const int a = c.node_ang[q];
                TOMO_REQUIRE(a >= 0 && a < A && !seen[a], "node_ang must be a permutation of the angles");
                seen[a] = 1;
            }
        }
        TOMO_REQUIRE(c.seg_row_ptr[0] == 0 && c.seg_row_ptr[M] == N, "seg_row_ptr must span the rows");
        for (int m = 0; m < M; ++m)
            TOMO_REQUIRE(c.seg_row_ptr[m + 1] > c.seg_row_ptr[m], "every segment needs at least one row");
        std::vector<int32_t> adj(c.adj, c.adj + (size_t)M * M);
        for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b)
                TOMO_REQUIRE(adj[(size_t)a * M + b] == adj[(size_t)b * M + a] && (a != b || !adj[(size_t)a * M + a]),
                             "adj must be symmetric with an empty diagonal");
        std::vector<int> dist, first;
        relay_tables(M, adj, dist, first);
        int max_lag = 0;
        for (int v : dist) {
            TOMO_REQUIRE(v >= 0, "the message graph must be connected");
            max_lag = std::max(max_lag, v - 1);
        }
        TOMO_REQUIRE(max_lag <= 125, "graph diameter too large");

        auto* h = new Dadmm();
        try {
            h->g = g;
            h->N = N;
            h->B = c.n_bins;
            h->A = A;
            h->S = c.S;
            h->M = M;
            TOMO_REQUIRE(c.max_stale >= 0 && c.max_stale <= 64, "max_stale must be in [0, 64]");
            h->max_stale = c.max_stale;
            // the ring also keeps node 0's previous view for the change statistic, and
            // max_stale older versions for nodes that lost messages (consensus: one exchange)
            h->D = cons ? 1 : max_lag + 2 + c.max_stale;
            h->variant = c.variant;
            h->E1 = c.E1;
            h->E2 = c.E2;
            h->rho = c.rho;
            h->eta2 = c.eta2;
            h->km_k = c.km_k;
            h->km_iters = c.km_iters;
            h->jpeg_q = c.jpeg_quality;
            h->seed = c.seed;
            h->mode = c.mode;
            h->seg_row_ptr.assign(c.seg_row_ptr, c.seg_row_ptr + M + 1);
            h->home_q.assign(c.home_q, c.home_q + M);
            // kinds
            h->lag.assign((size_t)M * M, 0);
            h->kind.assign((size_t)M * M, 0);
            h->recv_cnt.assign((size_t)M * 3, 0);
            h->need.assign((size_t)M, 0);
            for (int m = 0; m < M; ++m) {
                TOMO_REQUIRE(h->home_q[m] >= 0 && h->home_q[m] <= 2, "home_q must be a DADMM_Q_* value");
                h->need[m] |= 1 << h->home_q[m];
            }
            for (int s = 0; s < M; ++s)
                for (int m = 0; m < M; ++m) {
                    int kd;
                    if (s == m) {
                        kd = h->home_q[m];
                        h->lag[(size_t)m * M + s] = 0;
                    } else {
                        const int f = first[(size_t)s * M + m];
                        kd = c.edge_q[(size_t)s * M + f];
                        TOMO_REQUIRE(kd >= 0 && kd <= 2, "edge_q must be a DADMM_Q_* value on every edge");
                        h->lag[(size_t)m * M + s] = (int8_t)(dist[(size_t)s * M + m] - 1);
                        h->recv_cnt[(size_t)s * 3 + kd] += 1;
                        h->need[s] |= 1 << kd;
                    }
                    h->kind[(size_t)m * M + s] = (int8_t)kd;
                }
            if (cons) {  // one hop: node j sends to its neighbours, each edge with its quantizer
                std::fill(h->recv_cnt.begin(), h->recv_cnt.end(), 0);
                std::vector<int32_t> nb_ptr(M + 1, 0), nb;
                for (int m = 0; m < M; ++m) h->need[m] = 1 << h->home_q[m];
                for (int m = 0; m < M; ++m) {
                    nb.push_back(m | (h->home_q[m] << 16));
                    for (int j = 0; j < M; ++j)
                        if (j != m && adj[(size_t)j * M + m]) {
                            const int kd = c.edge_q[(size_t)j * M + m];
                            TOMO_REQUIRE(kd >= 0 && kd <= 2, "edge_q must be a DADMM_Q_* value on every edge");
                            nb.push_back(j | (kd << 16));
                            h->recv_cnt[(size_t)j * 3 + kd] += 1;
                            h->need[j] |= 1 << kd;
                        }
                    nb_ptr[m + 1] = (int32_t)nb.size();
                }
                h->d_nb_ptr = device_upload(nb_ptr);
                h->d_nb = device_upload(nb);
            }
            bool any_km = false, any_jp = false;
            for (int m = 0; m < M; ++m) {
                any_km |= (h->need[m] >> 1) & 1;
                any_jp |= (h->need[m] >> 2) & 1;
                if ((h->need[m] >> 2) & 1)
                    TOMO_REQUIRE((cons || (h->seg_row_ptr[m + 1] - h->seg_row_ptr[m]) % 8 == 0) && N % 8 == 0,
                                 "JPEG segments need row counts and N that are multiples of 8");
            }
            if (any_km) TOMO_REQUIRE(c.km_k >= 1 && c.km_k <= kKmMaxK && c.km_iters >= 0, "bad K-means settings");
            if (any_jp) TOMO_REQUIRE(c.jpeg_quality >= 1 && c.jpeg_quality <= 100, "bad JPEG quality");
            for (int m = 0; m < M; ++m)
                TOMO_REQUIRE(std::isfinite(c.eta1[m]) && c.eta1[m] > 0.0, "eta1 must be positive");

            // angle list (node-major), rows = natural angle index
            std::vector<AngRow> angs(A);
            for (int q = 0; q < A; ++q) angs[q] = AngRow{c.node_ang[q], c.node_ang[q]};
            h->angs = angs;
            h->node_ang_ptr.assign(c.node_ang_ptr, c.node_ang_ptr + M + 1);
            h->d_angs = device_upload(angs);
            h->d_bk = device_upload(bp_list_consts(*g, angs));
            TOMO_REQUIRE(c.tune == DADMM_TUNE_WIDE || c.tune == DADMM_TUNE_AUTO || c.tune == DADMM_TUNE_NARROW ||
                             c.tune == DADMM_TUNE_PAIRS || c.tune == DADMM_TUNE_QUADS ||
                             c.tune == DADMM_TUNE_WIDE_PAIRS,
                         "unknown tune setting");
            TOMO_REQUIRE(c.tune != DADMM_TUNE_PAIRS || c.S % 2 == 0, "slice pairs need an even number of slices");
            TOMO_REQUIRE((c.tune != DADMM_TUNE_QUADS && c.tune != DADMM_TUNE_WIDE_PAIRS) || c.S % 4 == 0,
                         "slice quads need S divisible by 4");
            h->tune = c.tune;
            if (c.tune == DADMM_TUNE_NARROW) {
                h->bp_tile_x = kBpTileXNarrow;
                h->proj_bins4 = kProjItemBinsNarrow;
            }
            if (c.tune == DADMM_TUNE_PAIRS) {  // narrow backprojector tiles; both operators in slice pairs
                h->bp_tile_x = kBpTileXNarrow;
                h->bp_slices = h->proj_slices = 2;
            }
            if (c.tune == DADMM_TUNE_QUADS) h->proj_slices = 4;  // wide backprojector tiles
            if (c.tune == DADMM_TUNE_WIDE_PAIRS) {  // wide backprojector tiles in slice pairs
                h->bp_slices = 2;
                h->proj_slices = 4;
            }
            build_lists(*h);
            // tables
            std::vector<int32_t> seg_of_row(N);
            for (int m = 0; m < M; ++m)
                for (int i = h->seg_row_ptr[m]; i < h->seg_row_ptr[m + 1]; ++i) seg_of_row[i] = m;
            h->d_lag = device_upload(h->lag);
            h->d_kind = device_upload(h->kind);
            h->d_seg_of_row = device_upload(seg_of_row);
            std::vector<int32_t> need2(h->need);  // + the rows of every message (consensus: whole images)
            for (int m = 0; m < M; ++m) need2.push_back(cons ? N : h->seg_row_ptr[m + 1] - h->seg_row_ptr[m]);
            h->d_need = device_upload(need2);
            h->d_recv = device_upload(h->recv_cnt);
            h->d_home = device_upload(h->home_q);
            std::vector<float> eta(M);
            for (int m = 0; m < M; ++m) eta[m] = (float)c.eta1[m];
            h->d_eta1 = device_upload(eta);
            h->d_eta0 = device_upload(std::vector<float>(M, 0.f));
            std::vector<float> mx(g->A);
            for (int a = 0; a < g->A; ++a) mx[a] = (float)std::fmax(std::fabs(g->c[a]), std::fabs(g->s[a]));
            h->d_mx = device_upload(mx);
            // codec tasks, slice-major
            std::vector<SegTask> km, jp;
            long long jp_blocks = 0;
            h->km_index.assign((size_t)c.S * M, -1);
            h->jp_index.assign((size_t)c.S * M, -1);
            for (int sl = 0; sl < c.S; ++sl)
                for (int m = 0; m < M; ++m) {
                    SegTask t{sl, m, h->seg_row_ptr[m], h->seg_row_ptr[m + 1], 0, 0, 0, 0, 0};
                    if (cons) {  // node m's whole message image
                        t.r0 = 0;
                        t.r1 = N;
                        t.src_off = t.dst_off = ((long long)sl * M + m) * N * N;
                    } else {
                        t.src_off = t.dst_off = (long long)sl * N * N + (long long)t.r0 * N;
                    }
                    if ((h->need[m] >> 1) & 1) {
                        h->km_index[(size_t)sl * M + m] = (int)km.size();
                        km.push_back(t);
                    }
                    if ((h->need[m] >> 2) & 1) {
                        h->jp_index[(size_t)sl * M + m] = (int)jp.size();
                        t.blk0 = (int)jp_blocks;
                        t.word0 = jp_blocks * kEntropyWordsPerBlock + (long long)jp.size();  // + 1 word each
                        jp_blocks += (long long)((t.r1 - t.r0) / 8) * (N / 8);
                        jp.push_back(t);
                        h->max_jp_rows = std::max(h->max_jp_rows, t.r1 - t.r0);
                    }
                }
            h->d_km = device_upload(km);
            h->d_jp = device_upload(jp);
            h->n_km = (int)km.size();
            h->n_jp = (int)jp.size();
            prepare_codecs(c.km_k);
            // workspace layout
            size_t off = 0;
            auto take = [&](size_t bytes) {
                const size_t o = off;
                off = align256(off + bytes);
                return o;
            };
            const size_t SMn = (size_t)c.S * M;
            h->off_uT = take(sizeof(float) * (size_t)c.S * M * N * N);
            h->off_w = take(sizeof(float) * (size_t)c.S * M * N * N);
            h->off_resid = take(sizeof(float) * (size_t)c.S * A * c.n_bins);
            h->off_counters = take(sizeof(int) * (2 * (size_t)c.E1 + 2));
            h->off_lo = take(sizeof(unsigned) * SMn);
            h->off_hi = take(sizeof(unsigned) * SMn);
            h->off_nnz = take(sizeof(long long) * SMn);
            if (c.max_stale > 0)
                h->off_held = take(sizeof(int32_t) * (4 + (size_t)DADMM_MAX_LOSSY_ITERS * 2 * M * M));
            h->off_coefs = take(sizeof(int16_t) * 64 * (size_t)std::max(jp_blocks, 1LL));
            h->off_bits = take(sizeof(uint32_t) * ((size_t)jp_blocks * kEntropyWordsPerBlock + jp.size() + 1));
            h->off_dual = take(sizeof(double) * 3 * SMn * kDualPerNode);
            h->off_res = take(sizeof(double) * (size_t)c.S * kResPerSlice);
            h->off_stats = take(sizeof(double) * (size_t)kStatsCap * c.S * DADMM_NSTAT);
            h->off_status = take(sizeof(int) * 4);
            h->ws_bytes = off + 256;
            TOMO_CUDA(cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking));
            TOMO_CUDA(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
            TOMO_CUDA(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
        } catch (...) {
            free_dadmm(h);
            throw;
        }
        *out = reinterpret_cast<dadmm_t>(h);
    });
}

tomo_status dadmm_destroy(dadmm_t hh) {
    return guard([&] {
        if (hh) free_dadmm(as_dadmm(hh));
    });
}

int dadmm_ring_depth(dadmm_t hh) { return hh ? reinterpret_cast<Dadmm*>(hh)->D : 0; }

tomo_status dadmm_launch_shape(dadmm_t hh, int* bp_tile_x, int* bp_slices, int* proj_item_bins, int* proj_slices) {
    return guard([&] {
        Dadmm& h = *as_dadmm(hh);
        TOMO_REQUIRE(bp_tile_x && bp_slices && proj_item_bins && proj_slices, "output pointers must be non-NULL");
        *bp_tile_x = h.bp_tile_x;
        *bp_slices = h.bp_slices;
        *proj_item_bins = h.proj_bins4;
        *proj_slices = h.proj_slices;
    });
}

size_t dadmm_state_size(dadmm_t hh) {
    if (!hh) return 0;
    const Dadmm& h = *reinterpret_cast<Dadmm*>(hh);
    const size_t n = (size_t)h.N * h.N;
    return sizeof(float) * (2 * (size_t)h.S * h.M * n + x_values(h) + hist_values(h)) + sizeof(int32_t);
}

size_t dadmm_workspace_size(dadmm_t hh) { return hh ? reinterpret_cast<Dadmm*>(hh)->ws_bytes : 0; }

tomo_status dadmm_state_init(dadmm_t hh, const dadmm_state* st, tomo_stream_t stream) {
    return guard([&] {
        Dadmm& h = *as_dadmm(hh);
        check_device(*h.g);
        TOMO_REQUIRE(st && st->u && st->lam && st->xseg && st->hist && st->iter, "state pointers must be non-NULL");
        const size_t n = (size_t)h.N * h.N;
        cudaStream_t s = (cudaStream_t)stream;
        TOMO_CUDA(cudaMemsetAsync(st->u, 0, sizeof(float) * h.S * h.M * n, s));
        TOMO_CUDA(cudaMemsetAsync(st->lam, 0, sizeof(float) * h.S * h.M * n, s));
        TOMO_CUDA(cudaMemsetAsync(st->xseg, 0, sizeof(float) * x_values(h), s));
        TOMO_CUDA(cudaMemsetAsync(st->hist, 0, sizeof(float) * hist_values(h), s));
        TOMO_CUDA(cudaMemsetAsync(st->iter, 0, sizeof(int32_t), s));
        h.der_dirty = true;
        h.held_k = -1;
    });
}

tomo_status dadmm_state_modified(dadmm_t hh) {
    return guard([&] {
        Dadmm& h = *as_dadmm(hh);
        h.der_dirty = true;
        h.held_k = -1;  // held versions restart from the lossless ones at the next lossy call
    });
}

tomo_status dadmm_sync_status(dadmm_t hh, void* workspace, size_t workspace_bytes, tomo_stream_t stream) {
    tomo_status numeric = TOMO_OK;
    tomo_status rc = guard([&] {
        Dadmm& h = *as_dadmm(hh);
        check_device(*h.g);
        TOMO_REQUIRE(workspace != nullptr && workspace_bytes >= h.ws_bytes,
                     "workspace too small: need " + std::to_string(h.ws_bytes) + " bytes");
        const WsPtrs w = ws_ptrs(h, workspace);
        cudaStream_t st = (cudaStream_t)stream;
        if (workspace != h.ws_status_init) {  // no iteration has run on this workspace yet
            TOMO_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), st));
            h.ws_status_init = workspace;
            return;
        }
        int status = 0;
        TOMO_CUDA(cudaMemcpyAsync(&status, w.status, sizeof(int), cudaMemcpyDeviceToHost, st));
        TOMO_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), st));
        TOMO_CUDA(cudaStreamSynchronize(st));
        check_status_word(status, &numeric);
    });
    if (rc == TOMO_OK && numeric != TOMO_OK) {
        set_last_error("non-finite statistics");
        return numeric;
    }
    return rc;
}

}  // extern "C"

namespace tomo {

// the held-version table of a lossy call: row i = (versions held at iteration k0+i, at k0+i+1);
// refuses a mask under which a version read would have left the ring
// process-wide choices of the launch shapes, keyed by the device and the
// problem's shape (sizes, trig table, angle partition)
static std::mutex g_shape_mu;
// launch shapes: backprojector tile width and slices per item, projector item bins
struct Shape {
    int tile_x, slices, bins4, pslices;
};
static std::map<std::vector<long long>, Shape> g_shape_cache;

static std::vector<long long> shape_key(const Dadmm& h) {
    int dev = 0;
    TOMO_CUDA(cudaGetDevice(&dev));
    std::vector<long long> k = {dev, h.N, h.B, h.A, h.S, h.M, h.has_maps};
    uint64_t f = 1469598103934665603ULL;  // FNV-1a over the trig table, the angle list and the partition
    auto mix = [&](uint64_t v) {
        for (int b = 0; b < 8; ++b) {
            f ^= (v >> (8 * b)) & 0xFF;
            f *= 1099511628211ULL;
        }
    };
    for (int a = 0; a < h.g->A; ++a) {
        uint64_t u;
        std::memcpy(&u, &h.g->c[a], 8);
        mix(u);
        std::memcpy(&u, &h.g->s[a], 8);
        mix(u);
    }
    for (const AngRow& r : h.angs) mix((uint64_t)r.angle);
    for (int32_t v : h.node_ang_ptr) mix((uint64_t)v);
    k.push_back((long long)f);
    return k;
}

// The launch shapes of the problem (the autotuner). tune = 1: once per problem
// shape and process, at the first step, the candidate shapes are timed on the
// caller's stream (which this synchronizes): the projector's items (128 or 64
// bins per angle, and slice pairs when S is even) on the state's u into the
// residual buffer, then the backprojector's tiles (wide, narrow, and narrow
// slice pairs when S is even) as the Algorithm 2 step itself with every step
// size eta1 = 0, so that u is rewritten with its own values (and u^T with
// their transpose); each twice after a warm-up launch. The fastest shape of
// each operator is kept and cached. The residual buffer is rewritten by the
// first inner step before it is read again. tune = 0 / 2 / 3 keep the wide /
// narrow / slice-pair shapes set at create.
static void tune_shapes(Dadmm& h, const dadmm_state& st, const float* sino, const WsPtrs& w, cudaStream_t s) {
    h.tuned = true;
    if (h.tune != DADMM_TUNE_AUTO) return;
    const std::vector<long long> key = shape_key(h);
    Shape pick{0, 0, 0, 0};
    {
        std::lock_guard<std::mutex> lk(g_shape_mu);
        auto it = g_shape_cache.find(key);
        if (it != g_shape_cache.end()) pick = it->second;
    }
    if (!pick.tile_x) {
        std::vector<std::pair<int, int>> pj_c = {{kProjItemBins, 1}, {kProjItemBinsNarrow, 1}};  // bins, slices
        std::vector<std::pair<int, int>> bp_c = {{kBpTileXWide, 1}, {kBpTileXNarrow, 1}};        // tile, slices
        if (h.S % 2 == 0) {
            pj_c.push_back({kProjItemBins, 2});
            bp_c.push_back({kBpTileXNarrow, 2});
            bp_c.push_back({kBpTileXWide, 2});
        }
        if (h.S % 4 == 0) pj_c.push_back({kProjItemBins, 4});
        const int nc = (int)std::max(pj_c.size(), bp_c.size());
        std::vector<float> tp(nc, INFINITY), tb(nc, INFINITY);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        TOMO_CUDA(cudaEventCreate(&e0));
        cudaError_t ce = cudaEventCreate(&e1);
        if (ce != cudaSuccess) cudaEventDestroy(e0);
        TOMO_CUDA(ce);
        try {
            for (int c = 0; c < nc; ++c) {
                const bool has_pj = c < (int)pj_c.size(), has_bp = c < (int)bp_c.size();
                h.proj_bins4 = pj_c[std::min<size_t>(c, pj_c.size() - 1)].first;
                h.proj_slices = pj_c[std::min<size_t>(c, pj_c.size() - 1)].second;
                h.bp_tile_x = bp_c[std::min<size_t>(c, bp_c.size() - 1)].first;
                h.bp_slices = bp_c[std::min<size_t>(c, bp_c.size() - 1)].second;
                build_lists(h);
                ProjParams pp = proj_params(h, st, sino, w);
                if (pp.has_map) {  // this candidate's box height
                    const int rows = kProjRows / h.proj_slices;
                    pp.has_map = pp.has_mapT = make_image_map(&pp.map, st.u, h.N, h.S * h.M, rows) &&
                                               make_image_map(&pp.mapT, w.uT, h.N, h.S * h.M, rows);
                    pp.map_rows = rows;
                }
                pp.items = h.d_pitems;
                pp.n_items = h.n_pitems;
                pp.counter = w.counters;
                BpParams bp = bp_params(h, st, w);
                bp.items = h.d_bitems;
                bp.n_items = h.n_bitems;
                bp.counter = w.counters + 1;
                bp.view.eta1 = h.d_eta0;
                for (int op = 0; op < 2; ++op) {
                    if ((op == 0 && !has_pj) || (op == 1 && !has_bp)) continue;
                    auto run = [&]() {
                        TOMO_CUDA(cudaMemsetAsync(w.counters, 0, 2 * sizeof(int), s));
                        if (op == 0)
                            launch_project(pp, std::min(h.grid_proj, h.n_pitems), s, h.proj_slices);
                        else
                            launch_backproject_ustep(bp, std::min(h.grid_bp, h.n_bitems), s, h.bp_tile_x,
                                                     h.bp_slices);
                    };
                    run();  // warm-up
                    TOMO_CUDA(cudaEventRecord(e0, s));
                    run();
                    run();
                    TOMO_CUDA(cudaEventRecord(e1, s));
                    TOMO_CUDA(cudaEventSynchronize(e1));
                    TOMO_CUDA(cudaEventElapsedTime(op == 0 ? &tp[c] : &tb[c], e0, e1));
                }
            }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        h.der_dirty = true;  // u^T is rebuilt from u before the first iteration reads it
        const int bi = (int)(std::min_element(tb.begin(), tb.begin() + bp_c.size()) - tb.begin());
        const int pi = (int)(std::min_element(tp.begin(), tp.begin() + pj_c.size()) - tp.begin());
        pick = Shape{bp_c[bi].first, bp_c[bi].second, pj_c[pi].first, pj_c[pi].second};
        std::lock_guard<std::mutex> lk(g_shape_mu);
        g_shape_cache.emplace(key, pick);
    }
    if (pick.tile_x != h.bp_tile_x || pick.slices != h.bp_slices || pick.bins4 != h.proj_bins4 ||
        pick.pslices != h.proj_slices) {
        h.bp_tile_x = pick.tile_x;
        h.bp_slices = pick.slices;
        h.proj_bins4 = pick.bins4;
        h.proj_slices = pick.pslices;
        build_lists(h);
    }
}

static void build_held_table(Dadmm& h, int k0, int n_iters, const uint8_t* drop) {
    const int M = h.M, MM = M * M, D = h.D;
    if ((int)h.held.size() != MM || h.held_k != k0) {  // the lossless versions at k0
        h.held.assign(MM, 0);
        for (int m = 0; m < M; ++m)
            for (int sg = 0; sg < M; ++sg) h.held[m * M + sg] = std::max(0, k0 - (int)h.lag[m * M + sg]);
    }
    h.held_tab.assign((size_t)n_iters * 2 * MM, 0);
    std::vector<int32_t> next(MM);
    for (int i = 0; i < n_iters; ++i) {
        const int k = k0 + i;
        for (int m = 0; m < M; ++m)
            for (int sg = 0; sg < M; ++sg) {
                const int mi = m * M + sg;
                const int newest = k + 1 - (int)h.lag[mi];
                const bool lost = sg != m && drop[((size_t)i * M + sg) * M + m] != 0;
                next[mi] = (!lost && newest >= 1) ? newest : h.held[mi];
                const int v0 = h.held[mi], v1 = next[mi];
                const bool ok = (v0 < 1 || v0 >= k + 1 - D) && (v1 < 1 || v1 >= k + 2 - D) &&
                                (m != 0 || v0 < 1 || v0 >= k + 2 - D);
                TOMO_REQUIRE(ok, "lost messages would make node " + std::to_string(m) + " read a version of segment " +
                                     std::to_string(sg) + " older than the message ring (raise max_stale)");
            }
        std::memcpy(&h.held_tab[(size_t)i * 2 * MM], h.held.data(), sizeof(int32_t) * MM);
        std::memcpy(&h.held_tab[((size_t)i * 2 + 1) * MM], next.data(), sizeof(int32_t) * MM);
        h.held.swap(next);
    }
    h.held_k = k0 + n_iters;
    h.held_stale = false;
    for (int mi = 0; mi < MM; ++mi)
        h.held_stale |= h.held[mi] != std::max(0, h.held_k - (int)h.lag[mi]);
}

static tomo_status run_steps(dadmm_t hh, const dadmm_state* st, const float* sino, int n_iters,
                             const uint8_t* drop, void* workspace, size_t workspace_bytes, double* stats,
                             tomo_stream_t stream) {
    tomo_status numeric = TOMO_OK;
    tomo_status rc = guard([&] {
        Dadmm& h = *as_dadmm(hh);
        check_device(*h.g);
        if (drop) {
            TOMO_REQUIRE(h.max_stale > 0, "lossy steps need a handle created with max_stale > 0");
            TOMO_REQUIRE(n_iters <= DADMM_MAX_LOSSY_ITERS, "n_iters above DADMM_MAX_LOSSY_ITERS");
        }
        TOMO_REQUIRE(st && st->u && st->lam && st->xseg && st->hist && st->iter, "state pointers must be non-NULL");
        TOMO_REQUIRE(sino != nullptr, "sino is NULL");
        TOMO_REQUIRE(n_iters >= 0, "n_iters must be >= 0");
        TOMO_REQUIRE(((uintptr_t)st->u | (uintptr_t)st->lam | (uintptr_t)st->xseg | (uintptr_t)st->hist) % 16 == 0,
                     "state arrays must be 16-byte aligned");
        TOMO_REQUIRE(workspace != nullptr && workspace_bytes >= h.ws_bytes,
                     "workspace too small: need " + std::to_string(h.ws_bytes) + " bytes");
        if (n_iters == 0) return;
        cudaStream_t user = (cudaStream_t)stream;
        const WsPtrs w = ws_ptrs(h, workspace);
        int k0 = 0;
        if (stats || drop) {
            TOMO_CUDA(cudaMemcpyAsync(&k0, st->iter, sizeof(int), cudaMemcpyDeviceToHost, user));
            TOMO_CUDA(cudaStreamSynchronize(user));
        }
        if (drop) {  // the versions held at every iteration of this call, and the first one's index
            build_held_table(h, k0, n_iters, drop);
            TOMO_CUDA(cudaMemcpyAsync(w.held, &k0, sizeof(int32_t), cudaMemcpyHostToDevice, user));
            TOMO_CUDA(cudaMemcpyAsync(w.held + 4, h.held_tab.data(), sizeof(int32_t) * h.held_tab.size(),
                                      cudaMemcpyHostToDevice, user));
        }
        h.lossy = drop != nullptr;
        if (stats || workspace != h.ws_status_init) {  // the status word covers this call (or starts here)
            TOMO_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), user));
            h.ws_status_init = workspace;
        }
        // TMA descriptors of u and u^T; u^T is rebuilt from u when the state or the
        // workspace changed (or the caller reported writing u), then kept in step by the
        // u-step epilogue
        auto build_maps = [&]() {
            h.map_rows = kProjRows / h.proj_slices;
            return make_image_map(&h.map_u, st->u, h.N, h.S * h.M, h.map_rows) &&
                   make_image_map(&h.map_uT, w.uT, h.N, h.S * h.M, h.map_rows);
        };
        const bool maps = build_maps();
        if (maps != (h.has_maps != 0)) h.drop_graphs();
        h.has_maps = maps ? 1 : 0;
        auto refresh_ut = [&]() {  // u^T and w, from the state as it is
            if (h.der_dirty || h.der_u != st->u || h.der_ws != workspace) {
                if (maps) launch_transpose(st->u, w.uT, h.N, h.S * h.M, user);
                const ElemParams ep = elem_params(h, *st, w);
                const long long rows = (long long)h.S * h.M * h.N;
                wprep_kernel<<<(int)std::min<long long>(rows, 152 * 8), kElemThreads, 0, user>>>(
                    ep, h.variant == DADMM_VARIANT_CONSENSUS ? st->xseg : nullptr);
                TOMO_CUDA(cudaGetLastError());
                h.der_u = st->u;
                h.der_ws = workspace;
                h.der_dirty = false;
            }
        };
        refresh_ut();  // the autotuner's trials read u^T and w too
        if (!h.tuned) {
            tune_shapes(h, *st, sino, w, user);
            if (maps) build_maps();  // the chosen shape's box height
        }
        refresh_ut();
        if (h.mode == DADMM_MODE_BATCHED) {
            const std::vector<const void*> key = {st->u, st->lam, st->xseg, st->hist, st->iter, sino,
                                                  w.resid, (const void*)(uintptr_t)(h.lossy ? 1 : 0)};
            size_t gi = 0;
            while (gi < h.graphs.size() && h.graphs[gi].key != key) ++gi;
            if (gi < h.graphs.size()) {  // most recently used last
                std::rotate(h.graphs.begin() + gi, h.graphs.begin() + gi + 1, h.graphs.end());
            } else {
                if (h.graphs.size() >= kGraphCache) {
                    TOMO_CUDA(cudaGraphExecDestroy(h.graphs.front().exec));
                    h.graphs.erase(h.graphs.begin());
                }
                cudaGraph_t graph = nullptr;
                TOMO_CUDA(cudaStreamBeginCapture(h.own, cudaStreamCaptureModeThreadLocal));
                try {
                    enqueue_iteration(h, *st, sino, w, h.own);
                } catch (...) {
                    cudaStreamEndCapture(h.own, &graph);
                    if (graph) cudaGraphDestroy(graph);
                    throw;
                }
                TOMO_CUDA(cudaStreamEndCapture(h.own, &graph));
                cudaGraphExec_t exec = nullptr;
                cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
                cudaGraphDestroy(graph);
                TOMO_CUDA(e);
                h.graphs.push_back({key, exec});
            }
            cudaGraphExec_t gexec = h.graphs.back().exec;
            TOMO_CUDA(cudaEventRecord(h.ev_in, user));
            TOMO_CUDA(cudaStreamWaitEvent(h.own, h.ev_in, 0));
            for (int it = 0; it < n_iters; ++it) TOMO_CUDA(cudaGraphLaunch(gexec, h.own));
            TOMO_CUDA(cudaEventRecord(h.ev_out, h.own));
            TOMO_CUDA(cudaStreamWaitEvent(user, h.ev_out, 0));
        } else {
            for (int it = 0; it < n_iters; ++it) enqueue_iteration(h, *st, sino, w, user);
        }
        if (stats) {
            const int keep = std::min(n_iters, kStatsCap);
            std::vector<double> ring((size_t)kStatsCap * h.S * DADMM_NSTAT);
            int status = 0;
            TOMO_CUDA(cudaMemcpyAsync(ring.data(), w.stats, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost, user));
            TOMO_CUDA(cudaMemcpyAsync(&status, w.status, sizeof(int), cudaMemcpyDeviceToHost, user));
            TOMO_CUDA(cudaStreamSynchronize(user));
            const size_t per = (size_t)h.S * DADMM_NSTAT;
            for (int it = 0; it < n_iters; ++it) {
                if (it < n_iters - keep) {  // overwritten in the ring: report NaN
                    for (size_t q = 0; q < per; ++q) stats[(size_t)it * per + q] = NAN;
                    continue;
                }
                const int kk = k0 + it;
                std::memcpy(stats + (size_t)it * per, ring.data() + (size_t)(kk % kStatsCap) * per, sizeof(double) * per);
            }
            check_status_word(status, &numeric);
        }
    });
    if (rc == TOMO_OK && numeric != TOMO_OK) {
        set_last_error("non-finite statistics");
        return numeric;
    }
    return rc;
}

}  // namespace tomo

extern "C" {

tomo_status dadmm_step(dadmm_t hh, const dadmm_state* st, const float* sino, int n_iters, void* workspace,
                       size_t workspace_bytes, double* stats, tomo_stream_t stream) {
    // after lost messages some nodes still hold old versions at the next iteration: that
    // one iteration reads them (a lossless exchange brings every node up to date)
    tomo::Dadmm* h = hh ? tomo::as_dadmm(hh) : nullptr;
    if (h && h->held_stale && n_iters > 0 && st && st->iter) {
        int k0 = -1;
        if (cudaMemcpyAsync(&k0, st->iter, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess ||
            cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
            tomo::set_last_error("reading the iteration counter failed");
            return TOMO_ERR_CUDA;
        }
        if (k0 == h->held_k) {
            const std::vector<uint8_t> none((size_t)h->M * h->M, 0);
            tomo_status rc = tomo::run_steps(hh, st, sino, 1, none.data(), workspace, workspace_bytes, stats, stream);
            if (rc != TOMO_OK || n_iters == 1) return rc;
            return tomo::run_steps(hh, st, sino, n_iters - 1, nullptr, workspace, workspace_bytes,
                                   stats ? stats + (size_t)h->S * DADMM_NSTAT : nullptr, stream);
        }
        h->held_stale = false;  // the state moved on without this handle's lossy calls
    }
    return tomo::run_steps(hh, st, sino, n_iters, nullptr, workspace, workspace_bytes, stats, stream);
}

tomo_status dadmm_step_lossy(dadmm_t hh, const dadmm_state* st, const float* sino, int n_iters, const uint8_t* drop,
                             void* workspace, size_t workspace_bytes, double* stats, tomo_stream_t stream) {
    if (!drop) {
        tomo::set_last_error("drop is NULL");
        return TOMO_ERR_INVALID_ARG;
    }
    return tomo::run_steps(hh, st, sino, n_iters, drop, workspace, workspace_bytes, stats, stream);
}

tomo_status dadmm_set_profiling(dadmm_t hh, int enable) {
    return guard([&] {
        Dadmm& h = *as_dadmm(hh);
        check_device(*h.g);
        if (enable && h.pev.empty()) {
            h.pev.resize(h.num_phases() + 1);
            for (auto& e : h.pev) TOMO_CUDA(cudaEventCreate(&e));
        }
        h.profiling = enable != 0;
        h.drop_graphs();  // the next step re-captures with or without the event nodes
    });
}

int dadmm_num_phases(dadmm_t hh) { return hh ? reinterpret_cast<Dadmm*>(hh)->num_phases() : 0; }

tomo_status dadmm_phase_times(dadmm_t hh, float* ms, int n) {
    return guard([&] {
        Dadmm& h = *as_dadmm(hh);
        TOMO_REQUIRE(h.profiling && !h.pev.empty(), "profiling is not enabled");
        TOMO_REQUIRE(ms != nullptr, "ms is NULL");
        TOMO_CUDA(cudaEventSynchronize(h.pev.back()));
        const int np = std::min(n, h.num_phases());
        for (int i = 0; i < np; ++i) TOMO_CUDA(cudaEventElapsedTime(ms + i, h.pev[i], h.pev[i + 1]));
    });
}

tomo_status dadmm_home_view(dadmm_t hh, const dadmm_state* st, float* out, tomo_stream_t stream) {
    return guard([&] {
        Dadmm& h = *as_dadmm(hh);
        check_device(*h.g);
        TOMO_REQUIRE(st && st->hist && st->iter && out, "state and out must be non-NULL");
        if (h.variant == DADMM_VARIANT_CONSENSUS)
            cons_view_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>(st->xseg, out, h.N, h.S, h.M);
        else
            home_view_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>(st->hist, st->iter, h.d_seg_of_row, h.d_home,
                                                                      out, h.N, h.S, h.D);
        TOMO_CUDA(cudaGetLastError());
    });
}

}  // extern "C"
