// Host side of the TMA passes: tensor-map encoding (through the driver entry
// point, so the library needs no link against the driver library), the shared-
// memory plan of a unit, path selection and the process-wide options.
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "../../include/snlm.h"
#include "snlm_host.h"
#include "snlm_internal.h"

namespace snlm {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

struct Options {
    std::atomic<int> tma{0};
    std::atomic<long long> wait_us{2000000};
    std::atomic<long long> inject{0};
};
Options &options()
{
    static Options o;
    return o;
}

__device__ unsigned g_device_error;   // SNLM_ERR_TIMEOUT (negated) once a bounded wait gave up

CUtensorMapDataType map_dtype(int dtype)
{
    return dtype == DT_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                          : (dtype == DT_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
}

// Geometry and tensor map of a view whose units cover `span` consecutive positions
// of kWarpsPerCta lines. False when the view cannot be moved by tensor copies
// (unaligned base or stride, lines that are neither rows nor columns).
bool make_view(TmaView &v, CUtensorMap &map, const void *ptr, int dtype, long long line_step, long long elem_step,
               int n_lines, int N, int span)
{
    memset(&v, 0, sizeof(v));
    const int es = (int)dtype_size(dtype);
    if (!ptr || (reinterpret_cast<uintptr_t>(ptr) & 15) != 0 || span < 1)
        return false;
    v.dtype = dtype;
    v.esize = es;
    v.align = 16 / es;
    cuuint64_t dims[2], strides[1];
    cuuint32_t box[2], estr[2] = {1, 1};
    if (elem_step == 1) {
        const long long sb = line_step * es;
        if (line_step < 1 || sb % 16 != 0 || sb >= (1LL << 40))
            return false;
        const int full = span + v.align - 1;                 // worst-case alignment slack
        v.mode = TMA_ROWS;
        v.nb = div_up(full, 256);
        v.bw = (int)align_up((size_t)div_up(full, v.nb), (size_t)(128 / es));
        v.bh = 1;
        v.sw = v.nb * v.bw;
        v.sq = 1;
        v.bytes = kWarpsPerCta * v.nb * v.bw * es;
        dims[0] = (cuuint64_t)N;
        dims[1] = (cuuint64_t)n_lines;
        strides[0] = (cuuint64_t)sb;
        box[0] = (cuuint32_t)v.bw;
        box[1] = 1;
    } else if (line_step == 1) {
        const long long sb = elem_step * es;
        if (elem_step < 1 || sb % 16 != 0 || sb >= (1LL << 40))
            return false;
        v.mode = TMA_COLS;
        v.bw = v.align > kWarpsPerCta ? v.align : kWarpsPerCta;   // lines per box (16 bytes at least)
        v.nb = div_up(span, 256);
        v.bh = (int)align_up((size_t)div_up(span, v.nb), 8);
        v.sw = 1;
        v.sq = v.bw;
        v.bytes = v.nb * v.bh * v.bw * es;
        dims[0] = (cuuint64_t)n_lines;
        dims[1] = (cuuint64_t)N;
        strides[0] = (cuuint64_t)sb;
        box[0] = (cuuint32_t)v.bw;
        box[1] = (cuuint32_t)v.bh;
    } else {
        return false;
    }
    if (v.bw > 256 || v.bh > 256 || (v.bw * es) % 16 != 0)
        return false;
    v.smem = (int)align_up((size_t)v.bytes, 128);
    EncodeTiledFn fn = encode_tiled();
    if (!fn)
        return false;
    const CUresult r = fn(&map, map_dtype(dtype), 2, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int num_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t occupancy(int K, int dm, bool sure, int smem, int *n)
{
    switch (K) {
    case 0: return pass_tma_occupancy<0>(dm, sure, smem, n);
    case 1: return pass_tma_occupancy<1>(dm, sure, smem, n);
    case 2: return pass_tma_occupancy<2>(dm, sure, smem, n);
    case 3: return pass_tma_occupancy<3>(dm, sure, smem, n);
    case 4: return pass_tma_occupancy<4>(dm, sure, smem, n);
    case 5: return pass_tma_occupancy<5>(dm, sure, smem, n);
    case 6: return pass_tma_occupancy<6>(dm, sure, smem, n);
    case 7: return pass_tma_occupancy<7>(dm, sure, smem, n);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch(int K, const PassArgs &a, const TmaPass &t, int dm, bool sure, int grid, cudaStream_t st)
{
    switch (K) {
    case 0: return launch_pass_tma<0>(a, t, dm, sure, grid, st);
    case 1: return launch_pass_tma<1>(a, t, dm, sure, grid, st);
    case 2: return launch_pass_tma<2>(a, t, dm, sure, grid, st);
    case 3: return launch_pass_tma<3>(a, t, dm, sure, grid, st);
    case 4: return launch_pass_tma<4>(a, t, dm, sure, grid, st);
    case 5: return launch_pass_tma<5>(a, t, dm, sure, grid, st);
    case 6: return launch_pass_tma<6>(a, t, dm, sure, grid, st);
    case 7: return launch_pass_tma<7>(a, t, dm, sure, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

// CTAs per SM of one kernel instantiation and shared-memory size (cached).
struct OccKey {
    int dev, K, dm, sure, smem;
};
int cached_occupancy(int K, int dm, bool sure, int smem)
{
    static std::mutex mu;
    static std::vector<std::pair<OccKey, int>> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    for (auto &e : cache)
        if (e.first.dev == dev && e.first.K == K && e.first.dm == dm && e.first.sure == (int)sure &&
            e.first.smem == smem)
            return e.second;
    int n = 0;
    if (occupancy(K, dm, sure, smem, &n) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    cache.push_back({OccKey{dev, K, dm, (int)sure, smem}, n});
    return n;
}

}  // namespace

bool tma_enabled() { return options().tma.load() != 0; }

unsigned *device_error_word()
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<unsigned *>(p);
}

// Plan the pass for the TMA kernel: true (with *t and *grid filled) when every
// array the pass reads can be moved by tensor copies and a unit fits in shared
// memory; false otherwise (the gathering kernel runs the pass).
bool plan_pass_tma(int K, const PassArgs &a, int dm, bool sure, TmaPass *tp, int *grid_out)
{
    if (!tma_enabled() || a.n_lines < 1 || a.N < 1 || K < 0 || K > kMaxK)
        return false;
    TmaPass &t = *tp;
    memset(&t, 0, sizeof(t));
    const int S = a.S, T = tile_positions(S);
    const int nch = div_up(S, kRun);
    t.win_len = 32 * kRun + nch * kRun + 2 * K + kRun;
    const WarpLayout L = warp_layout(S, K, sure, false);   // the gathering kernel's per-warp rows
    t.LF = L.LF;
    t.LW = L.LW;
    t.LT = L.LT;
    t.per_warp = L.per_warp;
    if (!make_view(t.v[TMA_SRC], t.map[TMA_SRC], a.src.ptr, a.src.dtype, a.src.line_step, a.src.elem_step,
                   a.n_lines, a.N, t.win_len))
        return false;
    struct Tile {
        int idx;
        const void *ptr;
        int dtype;
        long long ls, es;
    } tiles[4] = {
        {TMA_DIN, sure ? a.delta_in : nullptr, DT_F32, a.out_line_step, a.out_elem_step},
        {TMA_BLEND, a.blend, DT_F32, a.out_line_step, a.out_elem_step},
        {TMA_RC, sure ? a.aux_rc.ptr : nullptr, DT_F32, a.aux_rc.line_step, a.aux_rc.elem_step},
        {TMA_F, sure && a.aux_rc.ptr ? a.aux_f.ptr : nullptr, a.aux_f.dtype, a.aux_f.line_step, a.aux_f.elem_step},
    };
    for (const Tile &tl : tiles) {
        if (!tl.ptr)
            continue;
        if (!make_view(t.v[tl.idx], t.map[tl.idx], tl.ptr, tl.dtype, tl.ls, tl.es, a.n_lines, a.N, T))
            return false;
        // the epilogue reads a tile view with the store loop's thread mapping
        if ((t.v[tl.idx].mode == TMA_ROWS) != (a.out_elem_step == 1))
            return false;
    }
    // shared memory: per-warp float layout | window stage 0 | stage 1 | tile inputs
    size_t off = align_up((size_t)t.per_warp * kWarpsPerCta * sizeof(float), 128);
    t.v[TMA_SRC].off = (int)off;
    off += (size_t)t.v[TMA_SRC].smem;
    t.win_off1 = (int)off;
    off += (size_t)t.v[TMA_SRC].smem;
    for (int i = TMA_DIN; i < TMA_ARRAYS; ++i)
        if (t.v[i].mode != TMA_NONE) {
            t.v[i].off = (int)off;
            off += (size_t)t.v[i].smem;
        }
    off += 128;                                            // run-time alignment of the base
    if (off > 227 * 1024)
        return false;
    t.smem = (int)off;
    const long long units = (long long)div_up(a.N, T) * div_up(a.n_lines, kWarpsPerCta);
    if (units >= (1LL << 31))
        return false;
    t.units = (int)units;
    const int occ = cached_occupancy(K, dm, sure, t.smem);
    const int sms = num_sms();
    if (occ < 1 || sms < 1)
        return false;
    const long long grid = (long long)occ * sms < units ? (long long)occ * sms : units;
    t.wait_ns = (unsigned long long)options().wait_us.load() * 1000ull;
    t.err = device_error_word();
    long long inj = options().inject.load();
    while (inj > 0 && !options().inject.compare_exchange_weak(inj, inj - 1)) {
    }
    t.inject = inj > 0 ? 1 : 0;
    *grid_out = (int)grid;
    return true;
}

cudaError_t launch_planned_tma(int K, const PassArgs &a, const TmaPass &t, int dm, bool sure, int grid,
                               cudaStream_t st)
{
    return launch(K, a, t, dm, sure, grid, st);
}

}  // namespace snlm

using namespace snlm;

extern "C" {

int snlm_set_option(int option, long long value)
{
    switch (option) {
    case SNLM_OPT_TMA:
        if (value != 0 && value != 1)
            return SNLM_ERR_ARG;
        options().tma.store((int)value);
        return SNLM_OK;
    case SNLM_OPT_WAIT_LIMIT_US:
        if (value < 1 || value > 60LL * 1000 * 1000)
            return SNLM_ERR_ARG;
        options().wait_us.store(value);
        return SNLM_OK;
    case SNLM_OPT_INJECT_WAIT_TIMEOUT:
        if (value < 0)
            return SNLM_ERR_ARG;
        options().inject.store(value);
        return SNLM_OK;
    default:
        return SNLM_ERR_ARG;
    }
}

long long snlm_get_option(int option)
{
    switch (option) {
    case SNLM_OPT_TMA: return options().tma.load();
    case SNLM_OPT_WAIT_LIMIT_US: return options().wait_us.load();
    case SNLM_OPT_INJECT_WAIT_TIMEOUT: return options().inject.load();
    default: return -1;
    }
}

int snlm_device_error(void *stream)
{
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return SNLM_ERR_CUDA;
    }
    unsigned v = 0;
    const unsigned zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_device_error, sizeof(v)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_device_error, &zero, sizeof(zero)) != cudaSuccess) {
        cudaGetLastError();
        return SNLM_ERR_CUDA;
    }
    return v ? -(int)v : SNLM_OK;
}

}  // extern "C"
