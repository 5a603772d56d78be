// rebuild.cu -- cell-list rebuild (Algorithm 1: "update the multi-level data structure",
// "construct Verlet neighbour list") for every instance of a batch at once: cell key per
// particle, per-cell histogram, exclusive scan, scatter, and the gather of the state into
// sorted order with cell-relative offsets; the gather also orders each cell by stored index,
// which makes the counting sort stable and deterministic.
#include "sph_internal.cuh"

namespace sph {

// ---- key + histogram ----
template <typename T, int D, bool ONE> __global__ void __launch_bounds__(BLOCK) k_hash(State<T> s, One one) {
    reset_scan_state(s);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int inst = ONE ? 0 : inst_of(s, i);
    const Grid& g = ONE ? one.g : s.grids[inst];
    int key;
    if (!live(s, inst, i)) {
        key = g.base[MAXL];                      // padding: the instance's dummy cell
    } else {
        const int l = level_of(g, s.H[i]);
        int cell[3] = {s.C[0][i] >> l, s.C[1][i] >> l, D == 3 ? s.C[2][i] >> l : 0};
        key = key_of(g, l, cell);
    }
    s.K[i] = key;
    atomicAdd(s.count + key, 1);
}

// ---- exclusive scan of the per-cell counts: three passes over tiles of SCAN_TILE cells ----
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;   // inclusive scan of warp totals
    }
    __syncthreads();
    total = warp_sums[(blockDim.x >> 5) - 1];
    int before = wid > 0 ? warp_sums[wid - 1] : 0;
    return before + x - v;
}

// relative: the counters were not reset since the previous rebuild, where the scatter left
// count[c] = cell_start[c+1]; the new per-cell count is count[c] - cell_start[c+1] (and is
// stored back into count for the down-sweep), so no pass over all cells resets them.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(int ncell, int* __restrict__ count,
                                                              const int* __restrict__ cell_start, bool relative,
                                                              int* __restrict__ bsum) {
    __shared__ int ws[32];
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < ncell) {
            int nk = count[base + k];
            if (relative) {
                nk -= cell_start[base + k + 1];
                count[base + k] = nk;
            }
            v += nk;
        }
    int total;
    block_exclusive_scan(v, ws, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_top(int nb, int ncell, int* __restrict__ bsum,
                                                           int* __restrict__ cell_start, unsigned* __restrict__ occ,
                                                           int nocc) {
    __shared__ int ws[32];
    for (int t = threadIdx.x; t < nocc * OCCW; t += blockDim.x) occ[t] = 0u;   // rebuilt by the gather
    int base = threadIdx.x * SCAN_ITEMS;
    int loc[SCAN_ITEMS];
    int v = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        loc[k] = (base + k < nb) ? bsum[base + k] : 0;
        v += loc[k];
    }
    int total;
    int ex = block_exclusive_scan(v, ws, total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < nb) bsum[base + k] = ex;
        ex += loc[k];
    }
    if (threadIdx.x == 0) cell_start[ncell] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(int ncell, int* __restrict__ count,
                                                            const int* __restrict__ bsum,
                                                            int* __restrict__ cell_start) {
    __shared__ int ws[32];
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int loc[SCAN_ITEMS];
    int v = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        loc[k] = (base + k < ncell) ? count[base + k] : 0;
        v += loc[k];
    }
    int total;
    int ex = block_exclusive_scan(v, ws, total) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < ncell) {
            cell_start[base + k] = ex;
            count[base + k] = ex;    // scatter cursor
        }
        ex += loc[k];
    }
}

// ---- the step's scan in one pass: decoupled look-back ----
// Every block takes the next tile by ticket (so all tiles before it are running or done),
// computes its counts (relative: count[c] - cell_start[c+1], the previous scatter having left
// count[c] = cell_start[c+1]) and their sum, publishes the sum, then walks back over the
// preceding tiles' words (32 at a time, one per lane of its first warp) until it meets a
// published inclusive prefix, publishes its own
// inclusive prefix and writes cell_start and the scatter cursors of its cells.  A tile reads
// the old cell_start[c+1] of its last cell (the next tile's first) before it publishes its
// sum, and the next tile writes it only after it has seen that sum, so the read comes first.
// Spins are bounded: a tile that waits too long records ST_SCAN and goes on (the walks and the
// gather clamp every cell range, so the step stays in bounds; the host reports the error).
constexpr unsigned long long TS_AGG = 1ull << 62, TS_PRE = 2ull << 62, TS_VAL = 0xffffffffull;
constexpr int SCAN_SPIN_LIMIT = 1 << 20;

template <typename T> __global__ void __launch_bounds__(SCAN1_THREADS) k_scan_onepass(State<T> s) {
    __shared__ int ws[32];
    __shared__ int sh_tile, sh_prefix;
    if (threadIdx.x == 0) sh_tile = atomicAdd(s.ticket, 1);
    __syncthreads();
    const int tile = sh_tile;
    const int ncell = s.ncell;
    // occupancy words are rebuilt by the gather
    for (int t = tile * SCAN1_THREADS + threadIdx.x; t < s.nocc * OCCW; t += gridDim.x * SCAN1_THREADS) s.occ[t] = 0u;
    const int base = tile * SCAN1_TILE + threadIdx.x * SCAN1_ITEMS;
    int loc[SCAN1_ITEMS];
    int v = 0;
#pragma unroll
    for (int k = 0; k < SCAN1_ITEMS; ++k) {
        loc[k] = 0;
        if (base + k < ncell) loc[k] = s.count[base + k] - s.cell_start[base + k + 1];
        v += loc[k];
    }
    int agg;
    int ex = block_exclusive_scan(v, ws, agg);
    if (threadIdx.x < 32) {   // warp 0: publish, then look back 32 tiles at a time
        const int lane = threadIdx.x;
        if (tile == 0) {
            if (lane == 0) {
                atomicExch(s.tstate, TS_PRE | (unsigned)agg);
                sh_prefix = 0;
            }
        } else {
            if (lane == 0) atomicExch(s.tstate + tile, TS_AGG | (unsigned)agg);
            int prefix = 0, top = tile - 1, spins = 0;
            while (true) {
                const int p = top - lane;
                // before tile 0: an inclusive prefix of 0
                unsigned long long w = 2ull << 62;
                if (p >= 0) w = *reinterpret_cast<volatile unsigned long long*>(s.tstate + p);
                const unsigned flag = (unsigned)(w >> 62);
                const unsigned pre = __ballot_sync(0xffffffffu, flag == 2u);
                const unsigned none = __ballot_sync(0xffffffffu, flag == 0u);
                const int first = pre ? __ffs(pre) - 1 : 32;            // nearest inclusive prefix
                const unsigned need = first >= 31 ? 0xffffffffu : ((2u << first) - 1u);
                if (none & need) {                                      // a word it needs is not out yet
                    if (++spins >= SCAN_SPIN_LIMIT) {
                        if (lane == 0) atomicOr(&s.ctrls[0].status, ST_SCAN);
                        break;
                    }
                    continue;
                }
                int val = lane <= first ? (int)(w & TS_VAL) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
                prefix += val;
                if (first < 32) break;
                top -= 32;
            }
            if (lane == 0) {
                atomicExch(s.tstate + tile, TS_PRE | (unsigned)(prefix + agg));
                sh_prefix = prefix;
            }
        }
    }
    __syncthreads();
    ex += sh_prefix;
#pragma unroll
    for (int k = 0; k < SCAN1_ITEMS; ++k) {
        if (base + k < ncell) {
            s.cell_start[base + k] = ex;
            s.count[base + k] = ex;    // scatter cursor
        }
        ex += loc[k];
    }
    if (base + SCAN1_ITEMS >= ncell && base < ncell) s.cell_start[ncell] = ex;   // the thread holding the last cell
}

// ---- scatter into cells (order inside a cell fixed afterwards) ----
template <typename T> __global__ void __launch_bounds__(BLOCK) k_scatter(State<T> s) {
    dep_launch();
    dep_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int key = s.K[i];
    // one atomic per cell present in the warp (sorted neighbours mostly share cells); each
    // lane takes the cursor plus its rank among the lanes of its cell
    const unsigned peers = __match_any_sync(__activemask(), key);
    const int lane = threadIdx.x & 31, lead = __ffs(peers) - 1;
    int pos = 0;
    if (lane == lead) pos = atomicAdd(s.count + key, __popc(peers));
    pos = __shfl_sync(peers, pos, lead) + __popc(peers & ((1u << lane) - 1u));
    if ((unsigned)pos < (unsigned)s.n) {
        s.perm[pos] = i;
        s.Ks[pos] = key;   // every slot of a cell has the cell's key, whichever particle lands there
    }
}

// ---- per cell: order by stored index (stable sort), reset the count for the next rebuild ----
__global__ void __launch_bounds__(BLOCK) k_cellsort(int ncell, int n, const int* __restrict__ cell_start, int* perm,
                                                    int* __restrict__ count) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int s = cell_start[c], e = cell_start[c + 1];
    if (s < 0 || e > n) e = s;   // defensive: never index outside perm
    for (int a = s + 1; a < e; ++a) {
        int v = perm[a], b = a - 1;
        while (b >= s && perm[b] > v) {
            perm[b + 1] = perm[b];
            --b;
        }
        perm[b + 1] = v;
    }
    count[c] = 0;
}

// ---- gather into sorted order + cell-relative offsets ----
// The scatter fills each cell's slots in arbitrary order; slot k of cell c takes the particle
// whose stored index has rank (k - start_c) among the cell's particles, which makes the
// counting sort stable.  Usually a cell's particles were consecutive in the stored order (it
// is the previous step's sorted order), and the rank is found from the cell's minimum.
template <typename T, int D, bool ONE> __global__ void __launch_bounds__(BLOCK) k_gather(State<T> s, One one) {
    dep_launch();
    dep_wait();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.n) return;
    int i = s.perm[k];
    const int key = s.Ks[k];
    if ((unsigned)i >= (unsigned)s.n || (unsigned)key >= (unsigned)s.ncell) {
        // defensive: a broken permutation is reported, not followed
        atomicOr(&s.ctrls[0].status, ST_NONFINITE);
        return;
    }
    {
        const int c0s = max(s.cell_start[key], 0), c0e = min(s.cell_start[key + 1], s.n);
        const int m = c0e - c0s, r = k - c0s;
        if (m > 1 && r >= 0 && r < m) {
            int mn = INT_MAX, mx = INT_MIN;
            for (int t = c0s; t < c0e; ++t) {
                const int v = s.perm[t];
                mn = min(mn, v);
                mx = max(mx, v);
            }
            if (mx - mn + 1 == m) {
                i = mn + r;
            } else {
                for (int t = c0s; t < c0e; ++t) {
                    const int v = s.perm[t];
                    int below = 0;
                    for (int u = c0s; u < c0e; ++u) below += s.perm[u] < v;
                    if (below == r) i = v;
                }
            }
        }
        s.sperm[k] = i;
    }
    int c[3] = {0, 0, 0};
    T o[3] = {T(0), T(0), T(0)};
    const T h = s.H[i];
    const unsigned meta = s.G[i];
    Vec4<T> vh;
    vh.x = s.V[0][i];
    vh.y = s.V[1][i];
    vh.z = D == 3 ? s.V[2][i] : T(0);
    vh.w = h;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        c[a] = s.C[a][i];
        o[a] = s.O[a][i];
        s.Cs[a][k] = c[a];
        s.Os[a][k] = o[a];
    }
    s.VH[k] = vh;
    s.IDs[k] = s.ID[i];
    const int inst = ONE ? 0 : inst_of(s, k);
    if (!live(s, inst, k)) return;               // padding slot (sorted last in its instance)
    const Grid& g = ONE ? one.g : s.grids[inst];
    const int l = level_of(g, h);
    int cell[3];
    T off[3];
    level_repr<T, D>(g, l, c, o, cell, off);
    Rec<T, D>::store(s.P, s.Ms, k, off, h, (meta & 255u) | ((unsigned)cell[0] << 8));
    if (s.occ) {   // the largest h of the particle's level in the occupancy cell holding it
        const int sh = g.osh;
        int ct[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) ct[a] = min((cell[a] << l) >> sh, g.od[a] - 1);
        const int w = g.occ_base + (ct[2] * g.od[1] + ct[1]) * g.od[0] + ct[0];
        // sorted neighbours share the cell and the level: one atomic per distinct pair in the
        // warp (positive floats order as their bits)
        const unsigned peers = __match_any_sync(__activemask(), ((unsigned long long)w << 4) | (unsigned)l);
        const unsigned hbits = __reduce_max_sync(peers, __float_as_uint(float_up<T>(h)));
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(s.occ + (size_t)w * OCCW + l, hbits);
    }
}

// ---- initial smoothing lengths h = h_t(x) of one instance ----
template <typename T, int D> __global__ void __launch_bounds__(BLOCK) k_init_h(State<T> s, int inst) {
    const int i = __ldg(s.inst_off + inst) + blockIdx.x * blockDim.x + threadIdx.x;
    if (!live(s, inst, i) || i >= __ldg(s.inst_off + inst + 1)) return;
    const Grid& g = s.grids[inst];
    int c[3] = {s.C[0][i], s.C[1][i], D == 3 ? s.C[2][i] : 0};
    T o[3] = {s.O[0][i], s.O[1][i], D == 3 ? s.O[2][i] : T(0)};
    double x[3];
    pos64<T, D>(g, c, o, x);
    s.H[i] = (T)sizing_h(s.sizs[inst], x);
}

// ---- batch re-packing: instance i's stored state moves from slot old_off[i] to its new offset
// s.inst_off[i] (the first move_n[i] slots).  Pass 0 copies the stored arrays into the sorted
// arrays (scratch here: the next gather rewrites them), pass 1 copies them back, so moves
// between overlapping ranges never read a slot that was already overwritten.
template <typename T, int D>
__global__ void __launch_bounds__(BLOCK) k_repack(State<T> s, const int* __restrict__ old_off,
                                                  const int* __restrict__ move_n, int pass) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.n) return;
    const int i = inst_of(s, k);
    const int r = k - __ldg(s.inst_off + i);
    if (r >= __ldg(move_n + i)) return;
    if (pass == 0) {
        const int src = __ldg(old_off + i) + r;
        Vec4<T> vh;
        vh.x = s.V[0][src];
        vh.y = s.V[1][src];
        vh.z = D == 3 ? s.V[2][src] : T(0);
        vh.w = s.H[src];
        for (int a = 0; a < D; ++a) {
            s.Cs[a][k] = s.C[a][src];
            s.Os[a][k] = s.O[a][src];
        }
        s.VH[k] = vh;
        s.Ms[k] = s.G[src];
        s.IDs[k] = s.ID[src];
    } else {
        const Vec4<T> vh = s.VH[k];
        const T vv[3] = {vh.x, vh.y, vh.z};
        for (int a = 0; a < D; ++a) {
            s.C[a][k] = s.Cs[a][k];
            s.O[a][k] = s.Os[a][k];
            s.V[a][k] = vv[a];
        }
        s.H[k] = vh.w;
        s.G[k] = s.Ms[k];
        s.ID[k] = s.IDs[k];
    }
}

template <typename T, int D> void launch_repack(const State<T>& s, const int* old_off, const int* move_n, cudaStream_t st) {
    if (s.n == 0) return;
    k_repack<T, D><<<div_up(s.n, BLOCK), BLOCK, 0, st>>>(s, old_off, move_n, 0);
    k_repack<T, D><<<div_up(s.n, BLOCK), BLOCK, 0, st>>>(s, old_off, move_n, 1);
}

template <typename T, int D> void launch_hash(const State<T>& s, const One* one, cudaStream_t st) {
    if (one) k_hash<T, D, true><<<div_up(s.n, BLOCK), BLOCK, 0, st>>>(s, *one);
    else k_hash<T, D, false><<<div_up(s.n, BLOCK), BLOCK, 0, st>>>(s, One());
}
void launch_scan(int ncell, int* count, int* cell_start, int* bsum, cudaStream_t st, unsigned* occ, int nocc,
                 bool relative) {
    int nb = div_up(ncell, SCAN_TILE);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, st>>>(ncell, count, cell_start, relative, bsum);
    k_scan_top<<<1, SCAN_THREADS, 0, st>>>(nb, ncell, bsum, cell_start, occ, nocc);
    k_scan_down<<<nb, SCAN_THREADS, 0, st>>>(ncell, count, bsum, cell_start);
}
template <typename T> void launch_scan_onepass(const State<T>& s, cudaStream_t st) {
    k_scan_onepass<T><<<div_up(s.ncell, SCAN1_TILE), SCAN1_THREADS, 0, st>>>(s);
}
template <typename T> void launch_scatter(const State<T>& s, cudaStream_t st, bool pdl) {
    launch_k(k_scatter<T>, div_up(s.n, BLOCK), BLOCK, st, pdl, s);
}
void launch_cellsort(int ncell, int n, const int* cell_start, int* perm, int* count, cudaStream_t st) {
    k_cellsort<<<div_up(ncell, BLOCK), BLOCK, 0, st>>>(ncell, n, cell_start, perm, count);
}
template <typename T, int D> void launch_gather(const State<T>& s, const One* one, cudaStream_t st, bool pdl) {
    if (one) launch_k(k_gather<T, D, true>, div_up(s.n, BLOCK), BLOCK, st, pdl, s, *one);
    else launch_k(k_gather<T, D, false>, div_up(s.n, BLOCK), BLOCK, st, pdl, s, One());
}
template <typename T, int D> void launch_init_h(const State<T>& s, int inst, cudaStream_t st) {
    k_init_h<T, D><<<div_up(s.n, BLOCK), BLOCK, 0, st>>>(s, inst);   // threads past the instance exit
}

#define SPH_INST(T, D)                                                    \
    template void launch_hash<T, D>(const State<T>&, const One*, cudaStream_t);        \
    template void launch_gather<T, D>(const State<T>&, const One*, cudaStream_t, bool);      \
    template void launch_init_h<T, D>(const State<T>&, int, cudaStream_t);  \
    template void launch_repack<T, D>(const State<T>&, const int*, const int*, cudaStream_t);
SPH_INST(float, 2)
SPH_INST(float, 3)
SPH_INST(double, 2)
SPH_INST(double, 3)
template void launch_scan_onepass<float>(const State<float>&, cudaStream_t);
template void launch_scan_onepass<double>(const State<double>&, cudaStream_t);
template void launch_scatter<float>(const State<float>&, cudaStream_t, bool);
template void launch_scatter<double>(const State<double>&, cudaStream_t, bool);

}  // namespace sph
