// noalloc.cu -- cell-list rebuild for callers that cannot allocate device memory.
//
// sph_cell_sort_noalloc computes the same cell keys, cell starts and stable permutation as the
// handle-based rebuild, but takes every input and output as caller-owned device pointers and
// keeps its only scratch (per-cell counts and the scan's block sums) in a fixed file-scope
// device array.  It never calls cudaMalloc, cudaFree or any allocating routine.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/sphmesh.h"
#include "sph_internal.cuh"

namespace sph {
namespace {

constexpr int NA_BSUM = SPH_NOALLOC_MAX_CELLS / SCAN_TILE;

// Scratch of every call on a device: SPH_NOALLOC_MAX_CELLS per-cell counters (also the scatter
// cursors) followed by the block sums of the scan.  Every GPU that loads the library holds
// this array (4 MiB + 1 KiB) until the process exits.  Host code must not use the symbol
// itself as a device address: the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) int g_na_scratch[SPH_NOALLOC_MAX_CELLS + NA_BSUM];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
int* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

sph_status na_fail(sph_status s, const char* fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);   // reported by sph_last_error()
    return s;
}

__global__ void __launch_bounds__(BLOCK) k_na_zero(int* __restrict__ p, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0;
}

template <int D>
__global__ void __launch_bounds__(BLOCK) k_na_hash(Grid g, int n, const double* __restrict__ x0,
                                                   const double* __restrict__ x1, const double* __restrict__ x2,
                                                   const float* __restrict__ h, int* __restrict__ key,
                                                   int* __restrict__ count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[3] = {x0[i], x1[i], D == 3 ? x2[i] : 0.0};
    int l = level_of(g, h[i]);
    int c[3], cell[3];
    float o[3], off[3];
    fine_of<float, D>(g, x, c, o);              // finest cell, then the level's cell (c >> l)
    level_repr<float, D>(g, l, c, o, cell, off);
    for (int a = 0; a < D; ++a) cell[a] = min(cell[a], g.dims[l][a] - 1);   // never past the level's grid
    int k = key_of(g, l, cell);
    key[i] = k;
    if ((unsigned)k < (unsigned)g.ncell) atomicAdd(count + k, 1);
}

__global__ void __launch_bounds__(BLOCK) k_na_scatter(int n, const int* __restrict__ key, int* __restrict__ count,
                                                      int* __restrict__ perm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int pos = atomicAdd(count + key[i], 1);
    if ((unsigned)pos < (unsigned)n) perm[pos] = i;
}

}  // namespace
}  // namespace sph

using namespace sph;

#pragma GCC visibility push(default)
extern "C" sph_status sph_cell_sort_noalloc(const sph_grid_info* grid, int64_t n, const double* x_dev,
                                            const double* y_dev, const double* z_dev, const float* h_dev,
                                            int32_t* key_dev, int32_t* cell_start_dev, int32_t* perm_dev,
                                            void* stream) {
    if (!grid) return na_fail(SPH_E_INVALID, "cell_sort_noalloc: NULL grid");
    if (grid->dim != 2 && grid->dim != 3) return na_fail(SPH_E_INVALID, "cell_sort_noalloc: dim must be 2 or 3");
    if (grid->levels < 1 || grid->levels > SPH_MAX_LEVELS)
        return na_fail(SPH_E_INVALID, "cell_sort_noalloc: levels out of range");
    const int cps = grid->cells_per_support;
    if (cps != 1 && cps != 2 && cps != 4) return na_fail(SPH_E_INVALID, "cell_sort_noalloc: cells_per_support must be 1, 2 or 4");
    if (grid->n_cells < 1 || grid->n_cells > SPH_NOALLOC_MAX_CELLS)
        return na_fail(SPH_E_INVALID, "cell_sort_noalloc: the grid has %lld cells; this entry point supports at most %d",
                       (long long)grid->n_cells, SPH_NOALLOC_MAX_CELLS);
    if (n < 0 || n > (int64_t)1 << 30) return na_fail(SPH_E_INVALID, "cell_sort_noalloc: n out of range");
    if (!cell_start_dev) return na_fail(SPH_E_INVALID, "cell_sort_noalloc: NULL cell_start");
    {   // the key of every cell must stay inside [0, n_cells): check the grid's own consistency
        int64_t base = 0;
        for (int l = 0; l < grid->levels; ++l) {
            if (grid->base[l] != base) return na_fail(SPH_E_INVALID, "cell_sort_noalloc: inconsistent grid bases");
            int64_t cells = 1;
            for (int a = 0; a < 3; ++a) {
                const int64_t d = grid->dims[l][a];
                if (d < 1 || d >= ((int64_t)1 << 23) || (a >= grid->dim && d != 1))
                    return na_fail(SPH_E_INVALID, "cell_sort_noalloc: grid dims out of range");
                cells *= d;
            }
            base += cells;
        }
        if (base != grid->n_cells) return na_fail(SPH_E_INVALID, "cell_sort_noalloc: grid dims do not add up to n_cells");
        // a particle of level l takes the level cell (finest cell >> l) of a finest cell clamped
        // into dims[0]: every coarser level must cover the finest grid shifted down by l
        for (int l = 1; l < grid->levels; ++l)
            for (int a = 0; a < grid->dim; ++a)
                if (grid->dims[l][a] < ((grid->dims[0][a] - 1) >> l) + 1)
                    return na_fail(SPH_E_INVALID, "cell_sort_noalloc: level %d does not cover the finest grid", l);
        if (!(grid->c0 > 0.0f)) return na_fail(SPH_E_INVALID, "cell_sort_noalloc: c0 must be positive");
    }
    if (n > 0 && (!x_dev || !y_dev || (grid->dim == 3 && !z_dev) || !h_dev || !key_dev || !perm_dev))
        return na_fail(SPH_E_INVALID, "cell_sort_noalloc: NULL input or output array");

    Grid g;
    std::memset(&g, 0, sizeof g);
    g.D = grid->dim;
    g.L = grid->levels;
    g.c0 = grid->c0;
    for (int a = 0; a < 3; ++a) g.origin[a] = grid->origin[a];
    for (int l = 0; l < MAXL; ++l) {
        g.c[l] = std::ldexp((double)grid->c0, l);
        g.inv_c[l] = 1.0 / g.c[l];
        g.thr[l] = grid->thr[l];
        for (int a = 0; a < 3; ++a) g.dims[l][a] = l < grid->levels ? (int)grid->dims[l][a] : 1;
        g.base[l] = l < grid->levels ? (int)grid->base[l] : (int)grid->n_cells;
    }
    g.base[MAXL] = (int)grid->n_cells;
    g.ncell = (int)grid->n_cells;
    g.sm = cps == 1 ? 0 : (cps == 2 ? 1 : 2);
    g.osh = grid->levels - 1 + g.sm;   // no occupancy grid here

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(SPH_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(SPH_E_INVALID, "cell_sort_noalloc: device %d unsupported", dev);
    int* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            // one-time set-up on this device (the current one): the device address of the array
            int* p = nullptr;
            e = cudaGetSymbolAddress((void**)&p, g_na_scratch);
            if (e != cudaSuccess) return na_fail(SPH_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_na_ptr[dev] = p;
        }
        scratch = g_na_ptr[dev];
    }
    int* count = scratch;
    int* bsum = scratch + SPH_NOALLOC_MAX_CELLS;
    cudaStream_t st = (cudaStream_t)stream;
    const int nn = (int)n, nc = g.ncell;

    k_na_zero<<<div_up(nc, BLOCK), BLOCK, 0, st>>>(count, nc);
    if (nn > 0) {
        if (g.D == 2) k_na_hash<2><<<div_up(nn, BLOCK), BLOCK, 0, st>>>(g, nn, x_dev, y_dev, z_dev, h_dev, key_dev, count);
        else k_na_hash<3><<<div_up(nn, BLOCK), BLOCK, 0, st>>>(g, nn, x_dev, y_dev, z_dev, h_dev, key_dev, count);
    }
    launch_scan(nc, count, cell_start_dev, bsum, st);
    if (nn > 0) k_na_scatter<<<div_up(nn, BLOCK), BLOCK, 0, st>>>(nn, key_dev, count, perm_dev);
    launch_cellsort(nc, nn, cell_start_dev, perm_dev, count, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(SPH_E_CUDA, "cell_sort_noalloc launch: %s", cudaGetErrorString(e));
    return SPH_OK;
}
#pragma GCC visibility pop
