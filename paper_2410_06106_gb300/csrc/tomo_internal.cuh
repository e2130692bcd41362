// Internal declarations shared by the translation units of libtomo.
// Everything here is library-private; the public ABI is include/tomo.h.
#pragma once

#include <cuda.h>  // CUtensorMap (TMA descriptors); the driver entry point is fetched at run time
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <list>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tomo.h"

namespace tomo {

// ------------------------------------------------------------------
// errors: every extern "C" entry point runs its body inside guard(), which
// converts a thrown Error (or any exception) into a status code and records
// the message for tomo_last_error().
// ------------------------------------------------------------------
struct Error {
    tomo_status code;
    std::string msg;
};

void set_last_error(const std::string& msg);
void clear_last_error();

[[noreturn]] void fail(tomo_status code, const std::string& msg);

#define TOMO_REQUIRE(cond, msg)                                                  \
    do {                                                                         \
        if (!(cond)) ::tomo::fail(TOMO_ERR_INVALID_ARG, std::string(msg));       \
    } while (0)

#define TOMO_CUDA(call)                                                          \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess)                                                   \
            ::tomo::fail(TOMO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class F>
tomo_status guard(F&& body) {
    try {
        clear_last_error();
        body();
        return TOMO_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(std::string("internal error: ") + e.what());
        return TOMO_ERR_CUDA;
    } catch (...) {
        set_last_error("internal error");
        return TOMO_ERR_CUDA;
    }
}

// ------------------------------------------------------------------
// geometry
// ------------------------------------------------------------------

// one (angle, sinogram row) pair of a selection: the angle indexes the
// geometry's trig table, the row is where its sinogram line is read/written
struct AngRow {
    int angle;
    int row;
};

// projector work item: na consecutive entries of an AngRow list that share
// the major axis, a run of 128 bins of each, the major-index range covering
// every ray of the item, processed in chunks of kProjRows rows/columns
struct ProjItem {
    int img;      // image index (units of N*N floats)
    int outb;     // output row base (added to AngRow::row)
    int ang0;     // first AngRow entry
    int na;       // angles in the item (1, 2 or 4)
    int b0;       // first bin
    int m_lo;     // first major index
    int nchunks;  // chunks of kProjRows major indices
    int nb;       // bins of each angle (kProjItemBins, or kProjItemBinsNarrow for 4 narrow angles)
};

// backprojector work item: one 64 x 64 pixel tile of one image, all the
// angles of an AngRow run
struct __align__(16) BpItem {
    int img;   // image index (units of N*N floats); also the u/lambda index in dADMM
    int sinb;  // sinogram row base (added to BpConst::row)
    int tx, ty;
    int ang0, na;
    int node, slice;  // dADMM epilogue only
};
static_assert(sizeof(BpItem) == 32, "BpItem is copied in 16-byte pieces");

constexpr int kProjThreads = 256;
constexpr int kProjRows = 32;    // rows per staged chunk (the TMA box height)
constexpr int kProjPitch = 256;  // staged columns per row (the TMA box width)
constexpr int kProjWMax = 252;   // max staged minor extent; + 3 for the 16-byte aligned start
constexpr int kProjMaxNa = 4;
constexpr int kProjStageFloats = kProjRows * kProjPitch;  // one 32 KB stage; two stages in flight

constexpr int kBpThreads = 128;
constexpr int kBpTileY = 64;  // tile height; the width is 64 (wide) or 32 (narrow)
constexpr int kBpTileXWide = 64, kBpTileXNarrow = 32;
constexpr int kProjItemBins = 128;     // bins of each angle of a projector item
constexpr int kProjItemBinsNarrow = 64;  // 4-angle items of the narrow shape
constexpr int kBpChunk = 32;  // angles staged per pass
constexpr int kBpWin = 96;    // window pairs per angle: 63 (|c| + |s|) + 6 < 96

constexpr int kBpStageFloat2 = kBpChunk * kBpWin;  // one slice's window stage; two stages in flight
constexpr int kBpSmem = 2 * kBpStageFloat2 * (int)sizeof(float2);  // per slice of an item

constexpr double kFix = 1099511627776.0;  // 2^40, fixed-point scale of positions

// ------------------------------------------------------------------
// per-angle operator constants, derived on the host in FP64 when a
// geometry is created and kept in a device table per geometry
// ------------------------------------------------------------------

// projector: ray b at major index m has minor coordinate b Db + m Dm + K0
// (2^-40); the trapezoid weights of its two candidate pixels are
// sat(wf0 - kappa F) and sat(wf1 + kappa F) (F = 1 + fraction), times h
struct ProjAngle {
    long long Db, Dm, K0;
    int dm25;      // Dm in 2^-25, for stepping inside a chunk
    float kappa;   // |major| / |minor|: the weight slope in minor-index units
    float wf0, wf1;
    float h;       // 1 / |major|
    int colmaj;    // 0: image rows are the major axis; 1: columns
};

// backprojector: pixel (i, j) sits at bin coordinate j C - i S + K (2^-40);
// weights of its two candidate bins sat(wf0 - gam F), sat(wf1 + gam F).
// Work lists carry one entry per (angle, sinogram row) of their angle list,
// 64 bytes, so that a chunk's entries are copied with 16-byte cp.async.
struct __align__(16) BpConst {
    long long C, S, K;
    int C25, S25;    // cos, sin in 2^-25: the steps of one pixel in x and y
    float gam;       // 1 / min(|c|, |s|) (capped at 2^20)
    float wf0, wf1;
    float h;         // 1 / max(|c|, |s|)
    int row;         // sinogram line of this entry (relative to the item's line base)
    int CX16, SY8;   // steps of 16 pixels in x and 8 in y, rounded once (2^-25)
    int pad;
};
static_assert(sizeof(BpConst) == 64, "BpConst is copied in 16-byte pieces");

struct Geometry {
    int N = 0, B = 0, A = 0;
    int device = -1;
    ProjAngle* d_ptab = nullptr;  // [A] projector constants
    std::vector<BpConst> hb;      // [A] backprojector constants (host; lists copy from here)
    int* d_status = nullptr;  // device status word of standalone operator calls (bit 4: a wait gave up)
    std::vector<double> c, s;
    // cached device work lists of standalone project/backproject calls: one device
    // allocation per (angle selection, batch), kept until the budget below forces
    // the least recently used out, so repeated calls allocate nothing
    struct Sel {
        std::vector<int32_t> key;
        uint64_t hash = 0;
        int batch = 0;
        void* d_block = nullptr;  // the four lists below, 256-byte aligned inside one allocation
        size_t bytes = 0;
        AngRow* d_angs = nullptr;
        BpConst* d_bk = nullptr;  // backprojector constants of the selection, in its order
        ProjItem* d_pitems = nullptr;
        int n_pitems = 0;
        BpItem* d_bitems = nullptr;
        int n_bitems = 0;
    };
    std::list<Sel> cache;  // most recently used last
    size_t cache_bytes = 0;
    long long list_allocs = 0, list_frees = 0;
    std::mutex mu;
};
constexpr size_t kSelCacheBytes = size_t(256) << 20;  // device bytes of cached work lists per geometry
constexpr size_t kSelCacheEntries = 4096;             // cached selections per geometry

// host: true when the rows of the image are the major (iteration) axis of
// rays at this angle, i.e. |cos| >= |sin| (same test as the device)
inline bool rows_major(double c, double s) { return std::abs(c) >= std::abs(s); }

// host: the backprojector constants of an angle list, in its order
std::vector<BpConst> bp_list_consts(const Geometry& g, const std::vector<AngRow>& angs);

// host builders of work lists (operators.cu)
// bins4: bins per angle of 4-angle projector items (kProjItemBins or
// kProjItemBinsNarrow); tile_x: backprojector tile width (kBpTileXWide or
// kBpTileXNarrow)
void build_proj_items(const Geometry& g, const std::vector<AngRow>& angs, int ang_begin,
                      int ang_count, int img, int outb, std::vector<ProjItem>& out,
                      int bins4 = kProjItemBins);
void build_bp_items(const Geometry& g, int ang_begin, int ang_count, int img, int sinb,
                    int node, int slice, std::vector<BpItem>& out, int tile_x = kBpTileXWide);

// launch parameters. map / mapT: TMA descriptors of the images [nimg][N][N]
// and of their transposes; items of steep rays (columns major) read mapT,
// the others map. Without a descriptor an item stages its band with
// cp.async instead.
struct ProjParams {
    CUtensorMap map;
    CUtensorMap mapT;
    const float* img;
    float* out;
    const float* sub;  // may be null
    const ProjItem* items;
    const AngRow* angs;
    const ProjAngle* ptab;
    int* counter;  // null: one block per item; else persistent work queue
    int* status;   // device error word (may be null)
    int n_items;
    int N, B;
    int has_map, has_mapT;
    int map_rows;  // box height of map / mapT; the kernel uses TMA only when it equals its chunk rows
    int prescale;  // 1: write h (h P u - sub), the input the backprojector stages
    // slice-group items (slices of one node share the rays' arithmetic): the
    // image index and output line offsets from one slice to the next
    int pair_img, pair_rows;
};

// TMA descriptor of nimg images [N][N] float32 at base with a box of
// kProjPitch columns x `rows` rows (kProjRows, or kProjRows / slices for
// slice groups); false when the layout cannot be described (unaligned base, N % 4)
bool make_image_map(CUtensorMap* map, const float* base, int N, int nimg, int rows = kProjRows);

struct BpView {  // dADMM epilogue (Algorithm 2 step)
    const float* eta1;        // [M]
    float* u;                 // [S][M][N][N]
    float* uT;                // [S][M][N][N] transposed copy kept in step with u (may be null)
    const float* w;           // [S][M][N][N] lambda_m^k - rho x_m^k, fixed during the inner steps
    float rho;
};

struct BpParams {
    const float* sino;  // lines r_a, or h_a r_a when prescaled (the projector's prescaled output)
    float* img;         // EPI_STORE target
    const BpItem* items;
    const BpConst* bk;    // constants of the items' angle list (BpItem::ang0 indexes it)
    int* counter;         // persistent work queue; null: block b takes item b only
    int* status;
    int n_items;
    int N, B;
    int prescaled;  // 1: sino lines already carry the factor h_a
    float beta;
    // slice-pair items (two slices of one node and tile, sharing positions and
    // weights): the second slice's image index and sinogram line offsets
    int pair_img, pair_rows;
    BpView view;
};

// slices: 1, or 2 / 4 for slice-group items (chunks of kProjRows / slices rows)
void launch_project(const ProjParams& p, int grid, cudaStream_t st, int slices = 1);
void launch_transpose(const float* in, float* out, int N, int nimg, cudaStream_t st);
// slices: 1, or 2 for slice-pair items (narrow tiles only)
void launch_backproject_store(const BpParams& p, int grid, cudaStream_t st, int tile_x = kBpTileXWide,
                              int slices = 1);
void launch_backproject_ustep(const BpParams& p, int grid, cudaStream_t st, int tile_x = kBpTileXWide,
                              int slices = 1);
int persistent_grid_project(int slices = 1);
int persistent_grid_backproject(bool ustep, int tile_x = kBpTileXWide, int slices = 1);

Geometry* as_geometry(tomo_geometry_t g);
void check_device(const Geometry& g);

// small helpers
template <class T>
T* device_upload(const std::vector<T>& v) {
    if (v.empty()) return nullptr;
    T* d = nullptr;
    TOMO_CUDA(cudaMalloc(&d, sizeof(T) * v.size()));
    TOMO_CUDA(cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return d;
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace tomo

namespace tomo {

// ------------------------------------------------------------------
// codecs (codecs.cu)
// ------------------------------------------------------------------
constexpr int kKmThreads = 384;  // 4 blocks of 12 warps per SM (40 registers)
constexpr int kKmMaxK = 32;
constexpr int kKmProbes = 64;

// where the segment of (slice, owner) lives and where its messages go; built
// by dadmm_create, read by the dADMM variants of the codec kernels
struct SegTask {
    int slice, owner;
    int r0, r1;        // rows of the segment
    int blk0;          // JPEG: first of the segment's 8x8 blocks in the coefficient buffer
    int pad;
    long long word0;   // JPEG: first word of the segment's entropy-coding bit buffer
    long long src_off; // first value of the segment in the codec's source array
    long long dst_off; // first value of its message within a quantizer plane
};

struct DadmmCodec {
    const float* xseg;    // the source values (segments: x~ [S][N][N]; consensus: v [S][M][N][N])
    float* hist;          // message planes: slot * slot_stride + kind * plane_stride + dst_off
    size_t plane_stride, slot_stride;
    const int32_t* iter;  // completed iterations k (messages belong to k+1)
    const SegTask* tasks;
    int n_tasks;
    int N, S, D;
    uint64_t seed;
    // JPEG only
    const unsigned* lo_key;  // [S][M] order-preserving keys of the segment min / max
    const unsigned* hi_key;
    int16_t* coefs;          // quantized blocks of every task, natural order
    uint32_t* bits;          // entropy-coding bit buffers of every task
    long long* jbytes;       // [S][M] entropy-coded message bytes
    int M;
};

// worst case of the baseline entropy coder: 8x8 block = DC code + extra
// (9 + 11 bits) + 63 AC codes + extra (16 + 10 bits), in 32-bit words
constexpr int kEntropyWordsPerBlock = 52;

void launch_kmeans_single(const float* in, long long n, int k, int iters, uint64_t key,
                          uint8_t* codes, float* cent, float* deq, double* obj, cudaStream_t st);
void launch_kmeans_dadmm(const DadmmCodec& p, int k, int iters, int task_begin, int task_count,
                         cudaStream_t st);
void launch_jpeg_single(const float* in, int rows, int cols, int quality, int16_t* coefs,
                        float* lohi, float* deq, long long* nnz, cudaStream_t st);
void launch_jpeg_dadmm(const DadmmCodec& p, int quality, int max_rows, int task_begin,
                       int task_count, cudaStream_t st);
void launch_jpeg_entropy_dadmm(const DadmmCodec& p, int task_begin, int task_count, cudaStream_t st);
size_t kmeans_smem(int kmax);
void jpeg_quant_table(int quality, int32_t* qt);  // host, natural order

// order-preserving map float -> unsigned (min/max with integer atomics)
__host__ __device__ inline unsigned float_key(float f) {
    unsigned u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(f);
#else
    std::memcpy(&u, &f, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float key_float(unsigned k) {
    unsigned u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, 4);
    return f;
#endif
}

__host__ __device__ inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// splitmix64 counter key of the K-means initialisation for (seed, slice, owner, iteration)
__host__ __device__ inline uint64_t kmeans_key(uint64_t seed, int slice, int owner, int iter) {
    const uint64_t ctr = ((uint64_t)(uint32_t)slice << 48) ^ ((uint64_t)(uint32_t)owner << 32) ^
                         (uint64_t)(uint32_t)iter;
    return mix64(seed ^ mix64(ctr + 0x9E3779B97F4A7C15ULL));
}

}  // namespace tomo
