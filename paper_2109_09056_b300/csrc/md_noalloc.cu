// md_noalloc.cu -- md_bin_sort_noalloc: the binning + stable cell-order
// permutation for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc/cudaFree are off limits --
// for example inside a framework whose caching allocator has reserved the
// device's memory and forbids side allocations, or in a latency-critical loop
// that must never hit the implicit device-wide synchronisation that
// cudaMalloc/cudaFree can cause.  Such a caller passes only its inputs and the
// output array; every intermediate lives in one file-scope device array of
// fixed size that the library carries (held on every GPU that loads the
// library, until the process exits).
//
// Limits: at most kMaxAtoms atoms and kMaxCells cells; larger requests are
// rejected with MD_ERR_ARG.  The per-cell ordering ranks each atom against
// every atom of its cell (one warp per cell), so a cell of m atoms costs
// O(m^2) work: fine at liquid densities (~20 per cell), slow for a dense
// cluster of thousands of atoms in one cell.  The array is shared by every
// call on a device and keeps the previous call's contents; the histogram part
// is cleared at the start of each call.  Two calls whose work overlaps on the
// GPU (different streams without ordering) race on the array.
#include <cmath>
#include <mutex>

#include "md_common.cuh"

namespace {

constexpr int64_t kMaxAtoms = 1 << 18;  // 262,144 atoms
constexpr int64_t kMaxCells = 1 << 17;  // 131,072 cells
// int32 words: cell[kMaxAtoms] | rank[kMaxAtoms] | slot[kMaxAtoms] |
//              count[kMaxCells] | start[kMaxCells + 1]
constexpr int64_t kWords = 3 * kMaxAtoms + 2 * kMaxCells + 1;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) int32_t g_noalloc_scratch[kWords];

struct Grid {
    double L[3];
    double inv[3];
    int32_t nc[3];
};

__global__ void k_na_bin(const double *__restrict__ x, int64_t n, Grid g,
                         int32_t *__restrict__ cell, int32_t *__restrict__ rank,
                         int32_t *__restrict__ count) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
    for (int d = 0; d < 3; ++d) {
        const double L = g.L[d];
        const double q = floor(__ddiv_rn(x[3 * i + d], L));
        double w = __dsub_rn(x[3 * i + d], __dmul_rn(L, q));
        if (w < 0.0) w = __dadd_rn(w, L);
        if (w >= L) w = __dsub_rn(w, L);
        int cd = __double2int_rz(__dmul_rn(w, g.inv[d]));
        c[d] = cd < 0 ? 0 : (cd > g.nc[d] - 1 ? g.nc[d] - 1 : cd);
    }
    const int32_t gc = (c[2] * g.nc[1] + c[1]) * g.nc[0] + c[0];
    cell[i] = gc;
    rank[i] = atomicAdd(&count[gc], 1);
}

__global__ void __launch_bounds__(1024) k_na_scan(const int32_t *__restrict__ count,
                                                  int32_t *__restrict__ start, int32_t ncell) {
    __shared__ int32_t wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int per = (ncell + 1023) / 1024;
    const int lo = min(ncell, tid * per), hi = min(ncell, lo + per);
    int32_t s = 0;
    for (int c = lo; c < hi; ++c) s += count[c];
    int32_t incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int32_t ws = wsum[lane];
        int32_t wi = ws;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        wsum[lane] = wi - ws;
    }
    __syncthreads();
    int32_t run = wsum[w] + incl - s;
    for (int c = lo; c < hi; ++c) {
        start[c] = run;
        run += count[c];
    }
    if (tid == 1023) start[ncell] = wsum[31] + incl;
}

__global__ void k_na_scatter(int64_t n, const int32_t *__restrict__ cell,
                             const int32_t *__restrict__ rank, const int32_t *__restrict__ start,
                             int32_t *__restrict__ slot) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    slot[start[cell[i]] + rank[i]] = (int32_t)i;
}

// One warp per cell: order the cell's atoms by their input index.
__global__ void k_na_order(int32_t ncell, const int32_t *__restrict__ start,
                           const int32_t *__restrict__ slot, int32_t *__restrict__ perm) {
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= ncell) return;
    const int32_t s0 = start[c], m = start[c + 1] - s0;
    for (int e = lane; e < m; e += 32) {
        const int32_t val = slot[s0 + e];
        int32_t rk = 0;
        for (int u = 0; u < m; ++u) rk += (slot[s0 + u] < val);
        perm[s0 + rk] = val;
    }
}

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device address of the static scratch on the current device, looked up once
// per device (the name alone is only a host-side stand-in for it).
int32_t *scratch_address(cudaError_t *err) {
    static std::mutex mu;
    static int32_t *addr[kMaxDevices] = {};
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= kMaxDevices) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        int32_t *p = nullptr;
        *err = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        addr[dev] = p;
    }
    return addr[dev];
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" md_status md_bin_sort_noalloc(const md_box *box, int64_t n, const double *x,
                                         double rs, int32_t *perm, void *stream) {
    using mdb::set_global_error;
    if (!box || !x || !perm) return set_global_error(MD_ERR_ARG, "md_bin_sort_noalloc: NULL argument");
    if (n < 1 || n > kMaxAtoms)
        return set_global_error(MD_ERR_ARG, "md_bin_sort_noalloc: n must be in 1..262144");
    if (!(rs > 0.0) || !std::isfinite(rs))
        return set_global_error(MD_ERR_ARG, "md_bin_sort_noalloc: rs must be positive");
    Grid g;
    int64_t ncell = 1;
    for (int d = 0; d < 3; ++d) {
        const double L = box->L[d];
        if (!std::isfinite(L) || !(L > 2.0 * rs))
            return set_global_error(MD_ERR_BOX_TOO_SMALL, "md_bin_sort_noalloc: box edge must exceed 2*rs");
        // checked in FP64 before the conversion: a huge L/rs must not wrap
        const double ncd = std::floor(L / rs);
        if (!(ncd <= (double)kMaxCells))
            return set_global_error(MD_ERR_ARG, "md_bin_sort_noalloc: more than 131072 cells");
        g.L[d] = L;
        g.nc[d] = (int32_t)ncd;
        g.inv[d] = (double)g.nc[d] / L;
        ncell *= g.nc[d];
    }
    if (ncell > kMaxCells)
        return set_global_error(MD_ERR_ARG, "md_bin_sort_noalloc: more than 131072 cells");
    if (!on_device(x) || !on_device(perm))
        return set_global_error(MD_ERR_ARG, "md_bin_sort_noalloc: x and perm must be device memory");
    cudaError_t e;
    int32_t *s = scratch_address(&e);
    if (!s) return set_global_error(MD_ERR_CUDA, std::string("md_bin_sort_noalloc: ") + cudaGetErrorString(e));
    int32_t *cell = s, *rank = s + kMaxAtoms, *slot = s + 2 * kMaxAtoms;
    int32_t *count = s + 3 * kMaxAtoms, *start = count + kMaxCells;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(count, 0, sizeof(int32_t) * (size_t)ncell, st);
    if (e == cudaSuccess) {
        k_na_bin<<<blocks(n, 256), 256, 0, st>>>(x, n, g, cell, rank, count);
        k_na_scan<<<1, 1024, 0, st>>>(count, start, (int32_t)ncell);
        k_na_scatter<<<blocks(n, 256), 256, 0, st>>>(n, cell, rank, start, slot);
        k_na_order<<<blocks(ncell * 32, 256), 256, 0, st>>>((int32_t)ncell, start, slot, perm);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return set_global_error(MD_ERR_CUDA, std::string("md_bin_sort_noalloc: ") + cudaGetErrorString(e));
    return MD_OK;
}
