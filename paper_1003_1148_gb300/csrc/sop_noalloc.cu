// Verlet-list builder for callers that cannot allocate device memory.
//
// sop_pairlist_build_noalloc runs the same cell-list rebuild as the streamed
// schedule (bounding box, cell histogram, scan, scatter, per-cell order, one
// warp per bead writing its sorted row) for one system, but every scratch
// buffer it needs lives in the file-scope array below instead of memory from
// cudaMalloc. The caller passes the inputs and the output rows.
//
// The array is a fixed 2.5 MiB that every GPU which loads this library keeps
// until the process exits. Each call reads its counters back and synchronises its
// stream. The array's device address is looked up once per device, by the
// first call on that device, with cudaGetSymbolAddress (host code cannot use
// the symbol itself: in host code it names a host-side stand-in, not device
// memory); that first call should come before any stream capture begins. All
// calls share the array, so calls whose work overlaps on the GPU race on it.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>
#include <string>

#include "sop_internal.h"

namespace {

constexpr int kMaxBeads = SOP_NOALLOC_MAX_BEADS;
constexpr int kMaxCells = 2 * kMaxBeads + 8;                    // the streamed builder's cell budget
constexpr int kScanTmp = (kMaxCells + sop::kScanTileElems - 1) / sop::kScanTileElems + 2;   // block sums of the cell scan

// Scratch layout, in 32-bit words; each block starts on a 16-byte boundary.
constexpr int align4(int w) { return (w + 3) / 4 * 4; }
constexpr int kOffSys = 0;                                      // [n] system id (all 0)
constexpr int kOffCellOf = kOffSys + align4(kMaxBeads);         // [n]
constexpr int kOffSorted = kOffCellOf + align4(kMaxBeads);      // float4 [n]
constexpr int kOffCellCnt = kOffSorted + 4 * kMaxBeads;         // [cells]
constexpr int kOffCellStart = kOffCellCnt + align4(kMaxCells);  // [cells + 1]
constexpr int kOffScan = kOffCellStart + align4(kMaxCells + 1); // [scan]
constexpr int kOffSegLo = kOffScan + align4(kScanTmp);          // float4
constexpr int kOffSegDims = kOffSegLo + 4;                      // int4
constexpr int kOffSegBase = kOffSegDims + 4;                    // int64 [1] first column
constexpr int kOffSegEnd = kOffSegBase + 2;                     // int64 [1] column limit
constexpr int kOffBeadLo = kOffSegEnd + 2;                      // [2] segment bead offsets
constexpr int kOffCellBase = kOffBeadLo + 2;                    // [2] segment cell offsets
constexpr int kOffCursor = kOffCellBase + 2;                    // [1]
constexpr int kOffStatus = kOffCursor + 1;                      // [1]
constexpr int kOffHalt = kOffStatus + 1;                        // [1]
constexpr int kOffUsed = kOffHalt + 1;                          // [1] entries after an all-pairs build
constexpr int kOffSegBox = align4(kOffUsed + 1);                // [8] bounding-box accumulator
constexpr int kOffBruteLo = kOffSegBox + 8;                     // [2] all-pairs build CTAs of the segment
constexpr int kOffDone = kOffBruteLo + 2;                       // [1] its CTAs done
constexpr int kWords = align4(kOffDone + 1);

static __device__ __align__(256) int32_t g_noalloc_scratch[kWords];

std::mutex g_mu;
int32_t *g_addr[64] = {};   // device address of the scratch array, per device

// Zero what must start at zero and write the one-segment tables.
__global__ void k_noalloc_init(int32_t *w, int n, int64_t cap) {
    const int stride = gridDim.x * blockDim.x;
    const int cells = 2 * n + 8;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) w[kOffSys + k] = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cells; k += stride) w[kOffCellCnt + k] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        w[kOffBeadLo] = 0;
        w[kOffBeadLo + 1] = n;
        w[kOffCellBase] = 0;
        w[kOffCellBase + 1] = cells;
        reinterpret_cast<int64_t *>(w + kOffSegBase)[0] = 0;
        reinterpret_cast<int64_t *>(w + kOffSegEnd)[0] = cap;
        w[kOffCursor] = 0;
        w[kOffStatus] = 0;
        w[kOffHalt] = 0;
        w[kOffSegBox + 0] = w[kOffSegBox + 1] = w[kOffSegBox + 2] = INT_MAX;
        w[kOffSegBox + 3] = w[kOffSegBox + 4] = w[kOffSegBox + 5] = INT_MIN;
        w[kOffSegBox + 6] = w[kOffSegBox + 7] = 0;
        w[kOffUsed] = 0;
        w[kOffBruteLo] = 0;
        w[kOffBruteLo + 1] = (n + sop::kBruteSliceBeads - 1) / sop::kBruteSliceBeads;
        w[kOffDone] = 0;
    }
}

sop_status scratch_address(int32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        sop::set_global_error(std::string("noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return SOP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            sop::set_global_error(std::string("noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return SOP_ERR_CUDA;
        }
        g_addr[dev] = static_cast<int32_t *>(p);
    }
    *out = g_addr[dev];
    return SOP_OK;
}

}  // namespace

extern "C" sop_status sop_pairlist_build_noalloc(const float *pos4, int32_t n, const int32_t *chain,
                                                 const int32_t *nat_row, const int32_t *nat_col, double pair_cut,
                                                 int32_t *row_start, int32_t *row_len, int32_t *col, int64_t cap,
                                                 int64_t *nnz, void *cuda_stream) {
    using namespace sop;
    if (n < 1 || n > kMaxBeads) {
        set_global_error("noalloc: n must be in [1, SOP_NOALLOC_MAX_BEADS = " + std::to_string(kMaxBeads) + "]");
        return SOP_ERR_INVALID_ARG;
    }
    if (!pos4 || !chain || !nat_row || !nat_col || !row_start || !row_len || !col || !nnz || cap < 0 ||
        cap > INT32_MAX || !(pair_cut > 0.0)) {
        set_global_error("noalloc: a pointer is NULL, cap is out of range or pair_cut <= 0");
        return SOP_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(pos4) & 15u) != 0) {
        set_global_error("noalloc: pos4 must be 16-byte aligned (float4 per bead)");
        return SOP_ERR_INVALID_ARG;
    }
    int32_t *w = nullptr;
    sop_status st = scratch_address(&w);
    if (st != SOP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    StepArgs sa;
    sa.topo.n = n;
    sa.topo.n_sys = 1;
    sa.topo.chain = chain;
    sa.topo.sys = w + kOffSys;
    sa.topo.nat_row = nat_row;
    sa.topo.nat_col = nat_col;
    sa.cut2_d = pair_cut * pair_cut;
    sa.cut2_f = (float)sa.cut2_d;
    sa.R = 1;
    sa.rep_status = w + kOffStatus;
    sa.halt = w + kOffHalt;

    DevCells cells;
    cells.n_seg = 1;
    cells.seg_bead_lo = w + kOffBeadLo;
    cells.seg_cell_base = w + kOffCellBase;
    cells.seg_lo = reinterpret_cast<float4 *>(w + kOffSegLo);
    cells.seg_dims = reinterpret_cast<int4 *>(w + kOffSegDims);
    cells.cell_of = w + kOffCellOf;
    cells.cell_cnt = w + kOffCellCnt;
    cells.cell_start = w + kOffCellStart;
    cells.sorted = reinterpret_cast<float4 *>(w + kOffSorted);
    cells.scan_tmp = w + kOffScan;
    cells.seg_box = w + kOffSegBox;
    cells.brute_cta_lo = w + kOffBruteLo;
    cells.brute_done = w + kOffDone;
    cells.brute_used = w + kOffUsed;
    cells.n_cells = 2 * (int64_t)n + 8;

    DevPairList pl;
    pl.start = row_start;
    pl.len = row_len;
    pl.col = col;
    pl.cursor = w + kOffCursor;
    pl.seg_base = reinterpret_cast<const int64_t *>(w + kOffSegBase);
    pl.seg_end = reinterpret_cast<const int64_t *>(w + kOffSegEnd);
    pl.cap = cap;

    SegRange rg;
    rg.g_lo = 0;
    rg.g_hi = 1;
    rg.b_lo = 0;
    rg.b_hi = n;
    rg.c_lo = 0;
    rg.c_hi = 2 * n + 8;
    rg.max_seg = n;
    rg.k_lo = 0;
    rg.k_hi = (n + kBruteSliceBeads - 1) / kBruteSliceBeads;

    k_noalloc_init<<<64, 256, 0, s>>>(w, n, cap);
    launch_rebuild(sa, cells, pl, reinterpret_cast<const float4 *>(pos4), nullptr, rg, s, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_global_error(std::string("noalloc: launch: ") + cudaGetErrorString(e));
        return SOP_ERR_CUDA;
    }
    int32_t out[4] = {0, 0, 0, 0};   // cursor, status, halt, entries of an all-pairs build
    e = cudaMemcpyAsync(out, w + kOffCursor, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_global_error(std::string("noalloc: ") + cudaGetErrorString(e));
        return SOP_ERR_CUDA;
    }
    *nnz = n <= kBruteMaxBeads ? out[3] : out[0];   // the all-pairs build leaves its cursor reset
    switch (out[1]) {
    case 0: return SOP_OK;
    case SOP_ERR_PAIRLIST_OVERFLOW:
        set_global_error("noalloc: the list outgrew cap, or a row held more than " + std::to_string(kRowCandidates) +
                         " candidates");
        return SOP_ERR_PAIRLIST_OVERFLOW;
    case SOP_ERR_NONFINITE:
        set_global_error("noalloc: a position is NaN or infinite, or no cell grid within the 2 n + 8 cell budget "
                         "covers the system at this pair_cut; every row is empty");
        return SOP_ERR_NONFINITE;
    default:
        set_global_error("noalloc: the rebuild stopped with status " + std::to_string(out[1]));
        return (sop_status)out[1];
    }
}
