// noalloc.cu -- a neighbour-pair search that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another library
// is capturing the stream into a graph, real-time loops that must not touch
// the allocator, or hosts whose device memory is owned by a framework with a
// fixed budget.  gld_pairs_noalloc serves them: the caller passes the
// positions and the output buffers, and the cell-list scratch lives in the
// file-scope array below, which every GPU that loads this library holds until
// the process exits (about 4.3 MB).
#include <cmath>
#include <mutex>

#include "gld.h"
#include "launch.h"

using namespace gld;

namespace {

constexpr int kMaxN = GLD_NOALLOC_MAX_N;
constexpr int kMaxCellsPerSide = 64;
constexpr int kMaxCells = kMaxCellsPerSide * kMaxCellsPerSide * kMaxCellsPerSide;
// cells per block of the cell-list scan: the chunk sums below are sized by
// the block size that launch_cell_build uses
constexpr int kChunk = kBatchCellChunk;
constexpr int kMaxChunks = (kMaxCells + kChunk - 1) / kChunk;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffSorted = 0;
constexpr size_t kOffNext = kOffSorted + align256(sizeof(float4) * kMaxN);
constexpr size_t kOffStart = kOffNext + align256(sizeof(int) * kMaxN);
constexpr size_t kOffCount = kOffStart + align256(sizeof(int) * (kMaxCells + 1));
constexpr size_t kOffHead = kOffCount + align256(sizeof(int) * kMaxCells);
constexpr size_t kOffChunkSum = kOffHead + align256(sizeof(int) * kMaxCells);
constexpr size_t kOffChunkOff = kOffChunkSum + align256(sizeof(int) * kMaxChunks);
constexpr size_t kOffCtrl = kOffChunkOff + align256(sizeof(int) * kMaxChunks);
constexpr size_t kScratchBytes = kOffCtrl + align256(sizeof(Ctrl));

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_addr[kMaxDevices] = {nullptr};

__global__ void set_int(int* p, int v) { *p = v; }

// Device address of g_scratch on the current device, looked up once per device.
cudaError_t scratch_address(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (unsigned char*)p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" gld_status gld_pairs_noalloc(const float* pos4, int32_t n, double box, double r_c, int32_t* pairs,
                                        int64_t cap, unsigned long long* count, void* stream)
{
    if (n < 1 || n > kMaxN || !pos4 || !count || (cap > 0 && !pairs) || cap < 0 || !(box > 0) || !(r_c > 0) ||
        r_c > 0.5 * box || ((uintptr_t)pos4 & 15))
        return GLD_E_INVAL;
    unsigned char* s = nullptr;
    if (scratch_address(&s) != cudaSuccess) return GLD_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // Cell geometry as in gld_create, with at most 64 cells per side.
    int nc = (int)std::floor(box / r_c);
    while (nc > 0 && box / nc < r_c * (1.0 + 1e-5)) --nc;
    const int ncap = (int)std::floor(std::cbrt(8.0 * n));
    if (nc > ncap) nc = ncap;
    if (nc > kMaxCellsPerSide) nc = kMaxCellsPerSide;
    if (nc < 3) nc = 1;
    const int ncells = nc * nc * nc;
    StepParams P{};
    P.n = n;
    P.n_pad = n;
    P.nc = nc;
    P.box = (float)box;
    P.half_box = 0.5f * P.box;
    P.inv_box = 1.0f / P.box;
    P.inv_cell = (float)(nc / box);
    P.rc2 = (float)(r_c * r_c);
    ParticleBuffers B{};
    B.ctrl = (Ctrl*)(s + kOffCtrl);
    B.pos_sorted = (float4*)(s + kOffSorted);
    const float4* src = (const float4*)pos4;  // read only by the cell build
    B.cell_next = (int*)(s + kOffNext);
    B.cell_start = (int*)(s + kOffStart);
    B.cell_count = (int*)(s + kOffCount);
    B.cell_head = (int*)(s + kOffHead);
    B.chunk_sum = (int*)(s + kOffChunkSum);
    B.chunk_off = (int*)(s + kOffChunkOff);
    B.ncells = ncells;
    // The array keeps the previous call's contents: reset what must start
    // empty (cell counts, list heads, the scan's completion counter, output).
    if (cudaMemsetAsync(B.cell_count, 0, sizeof(int) * ncells, st) != cudaSuccess ||
        cudaMemsetAsync(B.cell_head, 0xff, sizeof(int) * ncells, st) != cudaSuccess ||
        cudaMemsetAsync(B.ctrl, 0, sizeof(Ctrl), st) != cudaSuccess ||
        cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return GLD_E_CUDA;
    set_int<<<1, 1, 0, st>>>(B.cell_start + ncells, n);
    if (cudaGetLastError() != cudaSuccess) return GLD_E_CUDA;
    if (launch_cell_build(P, B, src, nullptr, st) != cudaSuccess) return GLD_E_CUDA;
    if (launch_pair_list(P, B, pairs, cap, count, st) != cudaSuccess) return GLD_E_CUDA;
    return GLD_OK;
}
