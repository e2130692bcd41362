// Forward projection for callers that must not allocate device memory.
//
// tomo_project keeps the work list of every angle selection it sees in device
// memory that the library allocates with cudaMalloc on first use. Some callers
// cannot allow that: code that runs while another thread captures a CUDA
// graph, code that must stay inside a fixed memory budget or a custom pool, or
// real-time loops that forbid device allocation after start-up. For them,
// tomo_project_noalloc runs the same projector kernel with its work list placed
// in a fixed array in the library's own device image (a file-scope __device__
// array, part of the module and loaded with it on every GPU that uses the
// library, held until the process exits). The call performs no cudaMalloc or
// cudaFree and uses no allocating library routine; it only copies the host-built
// work list into that array on the caller's stream.
#include "tomo_internal.cuh"

namespace tomo {

// capacity of the fixed work-list array: work items and (angle, row) entries
constexpr int kNoAllocMaxItems = 16384;
constexpr int kNoAllocMaxAngles = 8192;
constexpr size_t kNoAllocItemBytes = sizeof(ProjItem) * kNoAllocMaxItems;
constexpr size_t kNoAllocBytes = kNoAllocItemBytes + sizeof(AngRow) * kNoAllocMaxAngles;  // 576 KiB

static __device__ __align__(256) unsigned char g_noalloc_worklist[kNoAllocBytes];

// Device address of the array on the current device. In host code the symbol
// g_noalloc_worklist is only a host-side stand-in, so its address must be
// asked from the runtime, with the device current; a kernel handed the host
// symbol would fault or read the wrong memory. The address is looked up on
// every call (the lookup allocates nothing) rather than cached, so it stays
// right if the caller tears down and re-creates a device's context. The
// first lookup on a device may load the library's module there.
static unsigned char* noalloc_worklist_address() {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_worklist);
    if (e != cudaSuccess || p == nullptr)
        fail(TOMO_ERR_CUDA, std::string("cudaGetSymbolAddress(work-list array): ") + cudaGetErrorString(e));
    return static_cast<unsigned char*>(p);
}

}  // namespace tomo

using namespace tomo;

extern "C" {

tomo_status tomo_project_noalloc(tomo_geometry_t gh, const float* img, float* sino, const int32_t* angle_idx,
                                 int n_sel, int batch, const float* subtract, tomo_stream_t stream) {
    return guard([&] {
        Geometry* g = as_geometry(gh);
        check_device(*g);
        TOMO_REQUIRE(img && sino, "img and sino must be non-NULL");
        TOMO_REQUIRE(batch >= 1, "batch must be >= 1");
        TOMO_REQUIRE(n_sel >= 1, "n_sel must be >= 1");
        TOMO_REQUIRE(angle_idx || n_sel == g->A, "angle_idx NULL requires n_sel == n_angles");
        cudaStream_t st = (cudaStream_t)stream;
        // the work list is copied from host buffers that live only for this call, so the
        // copies must run now, not be recorded into a graph that replays them later
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        TOMO_CUDA(cudaStreamIsCapturing(st, &cap));
        TOMO_REQUIRE(cap == cudaStreamCaptureStatusNone,
                     "tomo_project_noalloc: the stream is capturing a CUDA graph; the call copies its work "
                     "list from host memory it does not keep, so it refuses to be captured");
        if (n_sel > kNoAllocMaxAngles)
            fail(TOMO_ERR_WORKSPACE, "tomo_project_noalloc: " + std::to_string(n_sel) +
                                         " angles exceed the fixed work-list capacity of " +
                                         std::to_string(kNoAllocMaxAngles));
        std::vector<AngRow> angs(n_sel);
        for (int q = 0; q < n_sel; ++q) {
            const int a = angle_idx ? angle_idx[q] : q;
            TOMO_REQUIRE(a >= 0 && a < g->A, "angle index " + std::to_string(a) + " out of range");
            angs[q] = AngRow{a, q};
        }
        std::vector<ProjItem> items;
        for (int k = 0; k < batch; ++k) build_proj_items(*g, angs, 0, n_sel, k, k * n_sel, items);
        if ((long long)items.size() > kNoAllocMaxItems)
            fail(TOMO_ERR_WORKSPACE, "tomo_project_noalloc: the work list needs " + std::to_string(items.size()) +
                                         " items, more than the fixed capacity of " +
                                         std::to_string(kNoAllocMaxItems) + " (reduce batch or n_sel)");
        unsigned char* base = noalloc_worklist_address();
        ProjItem* d_items = reinterpret_cast<ProjItem*>(base);
        AngRow* d_angs = reinterpret_cast<AngRow*>(base + kNoAllocItemBytes);
        // pageable sources: each copy has read its host buffer when it returns
        TOMO_CUDA(cudaMemcpyAsync(d_items, items.data(), sizeof(ProjItem) * items.size(), cudaMemcpyHostToDevice, st));
        TOMO_CUDA(cudaMemcpyAsync(d_angs, angs.data(), sizeof(AngRow) * angs.size(), cudaMemcpyHostToDevice, st));
        ProjParams p{};
        p.img = img;
        p.out = sino;
        p.sub = subtract;
        p.items = d_items;
        p.angs = d_angs;
        p.counter = nullptr;
        p.status = g->d_status;
        p.n_items = (int)items.size();
        p.N = g->N;
        p.B = g->B;
        p.ptab = g->d_ptab;
        p.prescale = 0;
        launch_project(p, p.n_items, st);
    });
}

}  // extern "C"
