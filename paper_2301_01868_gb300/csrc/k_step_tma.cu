// k_step_tma.cu -- the fused stream-collide-force update with TMA staging.
//
// Same arithmetic as k_fused_step (clbm_cell.cuh), organised for sm_103a:
// persistent CTAs, one per SM, walk tiles of TR x TJ cells.  For every tile
// one thread issues one TMA box per population: rows [i0 - max(c1,0),
// i0 + TR + max(-c1,0)) and the columns the pull reaches (8-column halo only
// where c2 != 0), so each population plane brings exactly the rows and
// columns its pull and its lagged read touch (about 1.33 x the tile for
// D2Q21), plus the tile's table rows by a bulk copy.  Every shared-memory
// offset of a pull is a compile-time constant.  Two kernels share this:
//
// k_fused_ws (default): a producer warp fills 3 to 8 stages (as many as
//   fit in shared memory); 16 consumer warps each update 32 cells of a tile
//   row and store straight to global memory; full / empty mbarriers per
//   stage, no CTA-wide barrier in the tile loop.  k_batch_ws runs the same
//   loop over the tiles of a batch, k_residual_ws the residual sums.
// k_fused_tma: one elected thread, two stages, CTA-wide barriers, and a
//   shared output tile written back by one TMA store; the CTA copies the
//   periodic ghost columns and the ragged tail from that tile.
//
// Cells next to a wall write the ghost values they supply (EdgeFill).  Waits
// on mbarriers are bounded: on time-out the kernel records an error code,
// the other warps give up at their next wait, and loads in flight land
// before the CTA exits.
#include <cuda.h>

#include <cstring>
#include <type_traits>

#include "clbm_batch.cuh"
#include "clbm_cell.cuh"
#include "clbm_f2.cuh"
#include "clbm_sync.cuh"

namespace clbm {

// Interior columns the TMA tile store writes: whole 16-byte chunks of a row
// only.  Cells in the remaining n2 - tma_store_cols columns store themselves.
template <typename S>
__host__ __device__ __forceinline__ constexpr int tma_store_cols(int n2) {
    return n2 - n2 % (16 / (int)sizeof(S));
}

// Shared-memory layout of one tile (elements of the storage type S).
// TRO: rows of a tile when not the default (the two-cells-per-thread update
// runs 12-row tiles so that it keeps 12 consumer warps per SM).
template <int Q, typename S, int TRO = 0>
struct TileGeom {
    // D2Q21: 8 rows for every storage type (16-bit tiles of 10 rows, 20
    // consumer warps, ran 4-6 % slower: the register file then holds 80
    // registers per thread and the kernel spills).  D2Q9 (about 80
    // registers): 12 rows, 24 consumer warps, measured 3.5 % faster than 8
    // rows (10: +0.4 %, 14: +2.5 %)
    static constexpr int TR = TRO ? TRO : (Q == 9 ? 12 : 8), TJ = 64, NT = TR * TJ;
    static constexpr int HX = 8;                                  // column halo where c2 != 0
    static constexpr int ALIGN = 128 / (int)sizeof(S);            // keep sub-tiles 128-B aligned
    __host__ __device__ static constexpr int iabs(int x) { return x < 0 ? -x : x; }
    __host__ __device__ static constexpr int rows(int a) { return TR + iabs(c1_of(a)); }
    __host__ __device__ static constexpr int width(int a) { return c2_of(a) == 0 ? TJ : TJ + 2 * HX; }
    __host__ __device__ static constexpr int row0(int a) { return c1_of(a) > 0 ? c1_of(a) : 0; }
    __host__ __device__ static constexpr int col0(int a) { return c2_of(a) == 0 ? 0 : HX; }
    __host__ __device__ static constexpr int size(int a) {
        return (rows(a) * width(a) + ALIGN - 1) / ALIGN * ALIGN;
    }
    __host__ __device__ static constexpr int off(int a) {
        int s = 0;
        for (int b = 0; b < a; ++b) s += size(b);
        return s;
    }
    __host__ __device__ static constexpr int shape(int a) { return iabs(c1_of(a)) * 2 + (c2_of(a) != 0); }
    static constexpr int BUF = off(Q);                            // elements per input buffer
    static constexpr int OUT = Q * TR * TJ;                       // elements of the output tile
    static constexpr int TABB = TR * Tab<Q>::S * 4;               // bytes of one table block
    // two input buffers, two output tiles, two table blocks, barriers, alignment slack
    static constexpr int SMEM = 2 * BUF * (int)sizeof(S) + 2 * OUT * (int)sizeof(S) + 2 * TABB + 64 + 128;
};

// Warp-specialised pipeline over the same tiles: STAGES input stages (boxes
// and table rows), one producer warp issuing TMA loads, TR x TJ / 32 consumer
// warps that each update 32 cells of a tile row and store them straight to
// global memory (128-byte row segments).  Full / empty mbarriers per stage
// replace every CTA-wide barrier of the tile loop.
// CPT: cells per consumer thread (2: neighbouring cells of a row in the two
// lanes of the packed F2 arithmetic, half as many consumer warps).
template <int Q, typename S, int CPT = 1, int TRO = 0>
struct PipeGeom {
    using G = TileGeom<Q, S, TRO>;
    static constexpr int CONSUMERS = G::NT / 32 / CPT;
    static constexpr int NTHREADS = CONSUMERS * 32 + 32;
    static constexpr int IN_BYTES = (G::BUF * (int)sizeof(S) + 127) / 128 * 128;
    static constexpr int STAGE_BYTES = IN_BYTES + (G::TABB + 127) / 128 * 128;
    // as many stages as fit in 220 KB of shared memory (2 to 8): the smaller
    // the stage (D2Q9, 16-bit storage), the more tiles are in flight, so every
    // configuration keeps about the same bytes on their way from HBM per SM
    static constexpr int FIT = (220 * 1024) / STAGE_BYTES;
    static constexpr int STAGES = FIT > 8 ? 8 : (FIT < 2 ? 2 : FIT);
    // per stage, a slot for the tile's descriptor when the producer publishes
    // it (batches: the lattice a tile belongs to comes from global memory)
    static constexpr int TILE_SLOT = 256;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 2 * STAGES * 8 + 16 + STAGES * TILE_SLOT + 128;
    static_assert(SMEM + 2048 <= 227 * 1024, "pipeline stages exceed shared memory");
};

// Tensor maps of both state buffers: per buffer, the 8 box shapes of the loads
// (|c1| = 0..3, c2 zero / nonzero) and the interior map of the tile store.
struct TmaMaps {
    CUtensorMap ld[2][8];
    CUtensorMap st[2];
    CUtensorMap ld12[2][8];   // the same load boxes for 12-row tiles (two cells per thread)
};

namespace {

__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store3(const CUtensorMap* map, int x, int y, int z, const void* src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map),
                 "r"(x), "r"(y), "r"(z), "r"(smem_addr(src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until at most one committed bulk store still reads shared memory.
__device__ __forceinline__ void bulk_wait_read1() {
    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int Q, typename S, typename C>
__device__ __forceinline__ void issue_tile(const TmaMaps& maps, int buf, int tile, int tiles_j,
                                           const StepArgs& a, unsigned char* sm_in, unsigned char* sm_tab,
                                           uint64_t* bar) {
    using G = TileGeom<Q, S>;
    constexpr int H = Lat<Q>::H;
    const int i0 = (tile / tiles_j) * G::TR, j0 = (tile % tiles_j) * G::TJ;
    const int nrows = a.n1 - i0 < G::TR ? a.n1 - i0 : G::TR;
    uint32_t bytes = (uint32_t)nrows * Tab<Q>::S * 4;
#pragma unroll
    for (int al = 0; al < Q; ++al) bytes += G::rows(al) * G::width(al) * (int)sizeof(S);
    mbar_expect(bar, bytes);
    S* in = (S*)sm_in;
#pragma unroll
    for (int al = 0; al < Q; ++al)
        tma_load3(in + G::off(al), &maps.ld[buf][G::shape(al)], j0 + GC - G::col0(al),
                  i0 + H - G::row0(al), al, bar);
    bulk_load(sm_tab, (const C*)a.tab + (size_t)i0 * Tab<Q>::S, (uint32_t)nrows * Tab<Q>::S * 4, bar);
}

template <int Q, typename S, typename C>
__global__ void __launch_bounds__((TileGeom<Q, S>::NT), 1)
    k_fused_tma(const __grid_constant__ TmaMaps maps, const StepArgs a, int src) {
    using G = TileGeom<Q, S>;
    using T = Tab<Q>;
    constexpr int H = Lat<Q>::H;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // round up to 128 bytes by pointer arithmetic (keeps the shared address space)
    unsigned char* const smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    unsigned char* const in_base = smem;
    S* const out_base = (S*)(smem + 2 * G::BUF * sizeof(S));
    unsigned char* const tab_base = smem + 2 * G::BUF * sizeof(S) + 2 * G::OUT * sizeof(S);
    uint64_t* const bar = (uint64_t*)(tab_base + 2 * G::TABB);
    int* const s_abort_p = (int*)(bar + 2);
#define s_abort (*s_abort_p)
    auto sm_in = [&](int b) { return in_base + b * (G::BUF * sizeof(S)); };
    auto sm_tab = [&](int b) { return tab_base + b * G::TABB; };

    const int tid = threadIdx.x;
    const int r = tid / G::TJ, cc = tid % G::TJ;
    const int tiles_j = (a.n2 + G::TJ - 1) / G::TJ;
    const int ntiles = ((a.n1 + G::TR - 1) / G::TR) * tiles_j;
    const Consts<C> k = Consts<C>::make(a.k);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int tile = blockIdx.x;
    int it = 0;
    bool next_issued = false;
    if (tid == 0 && tile < ntiles)
        issue_tile<Q, S, C>(maps, src, tile, tiles_j, a, sm_in(0), sm_tab(0), &bar[0]);
    for (; tile < ntiles; ++it, tile += gridDim.x) {
        const int buf = it & 1;
        const int next = tile + gridDim.x;
        next_issued = next < ntiles;
        if (tid == 0 && next_issued)
            issue_tile<Q, S, C>(maps, src, next, tiles_j, a, sm_in(buf ^ 1), sm_tab(buf ^ 1),
                                &bar[buf ^ 1]);
        if (!mbar_wait(&bar[buf], (it >> 1) & 1)) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        const int i0 = (tile / tiles_j) * G::TR, j0 = (tile % tiles_j) * G::TJ;
        const int i = i0 + r, j = j0 + cc;
        if (i < a.n1 && j < a.n2) {
            const RowTab<Q, C> tb{(const C*)sm_tab(buf) + r * T::S};
            const S* in = (const S*)sm_in(buf);
            Cell<Q, C> c;
            pull_cell<Q, C>(
                [&](int al, int dr, int dc) -> C {
                    return C(Store<S>::lds(in + G::off(al) + (r + G::row0(al) + dr) * G::width(al) +
                                           cc + G::col0(al) + dc));
                },
                tb, k, c);
            S* out = out_base + (it & 1) * G::OUT + r * G::TJ + cc;
            collide_emit<Q, C>(tb, c, k, [&](int al, C v) {
                Store<S>::st(out + al * (G::TR * G::TJ), v);
            });
            if (i < H || i >= a.n1 - H) {
                const EdgeFill<Q, S> ef{(S*)a.dst, (const typename Store<S>::C*)a.ghost, a.plane, a.ld, a.n1, a.n2, a.bc_lo,
                                        a.bc_hi, C(a.U0_lo), C(a.U0_hi), false, 1};
                ef.fill(i, j, out, G::TR * G::TJ, c.rho, c.Ut2);
            }
            if (i < H) {
                const int idx = i * a.n2 + j;
                ((C*)a.wall_rho)[idx] = c.rho;
                ((C*)a.wall_ut2)[idx] = c.Ut2;
            }
            if (i >= a.n1 - H) {
                const int idx = (H + (a.n1 - 1 - i)) * a.n2 + j;
                ((C*)a.wall_rho)[idx] = c.rho;
                ((C*)a.wall_ut2)[idx] = c.Ut2;
            }
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            // store this tile; the output tile of the previous one must be read
            // out before the next tile overwrites it (double-buffered)
            tma_store3(&maps.st[src ^ 1], j0, i0, 0, out_base + (it & 1) * G::OUT);
            bulk_wait_read1();
        }
        // Tiles at the periodic ends: the whole CTA copies, from the output
        // tile, the periodic ghost columns its cells supply and the ragged
        // tail the tile store leaves out (columns j < GC, and the last GC
        // columns, which hold every column past the last whole 16-byte chunk).
        if (j0 < GC || j0 + G::TJ > a.n2 - GC) {
            const int n2v = tma_store_cols<S>(a.n2);
            const int jend = j0 + G::TJ < a.n2 ? j0 + G::TJ : a.n2;
            const S* ob = out_base + (it & 1) * G::OUT;
            for (int e = tid; e < Q * G::TR * 2 * GC; e += G::NT) {
                const int x = e % (2 * GC), rr = (e / (2 * GC)) % G::TR, al = e / (2 * GC * G::TR);
                const int jj = x < GC ? x : a.n2 - 2 * GC + x;
                const int ii = i0 + rr;
                if (jj < j0 || jj >= jend || ii >= a.n1) continue;
                const C v = C(Store<S>::lds(ob + al * (G::TR * G::TJ) + rr * G::TJ + (jj - j0)));
                S* rowp = (S*)a.dst + al * a.plane + (long long)(ii + H) * a.ld;
                if (jj >= n2v) Store<S>::st(rowp + jj + GC, v);
                store_wrap<S, C>(rowp, jj, a.n2, v);
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        bulk_wait_all();
        if (s_abort) {
            atomicExch(a.err, 1);
            // let the loads that may still be in flight land before the CTA exits
            const int buf = it & 1;
            mbar_wait(&bar[buf], (it >> 1) & 1);
            if (next_issued) mbar_wait(&bar[buf ^ 1], ((it + 1) >> 1) & 1);
        }
    }
#undef s_abort
}

// What a consumer needs of the lattice a tile belongs to.
template <typename S>
struct WsLattice {
    S* dst;                 // state buffer written (row 0, column 0)
    const void* ghost;        // compute type
    void* wall_rho;
    void* wall_ut2;
    long long plane;
    int ld, n1, n2, bc_lo, bc_hi;
    double U0_lo, U0_hi;
};

// One consumer thread's cell (i0 + r, j0 + cc) of a tile staged in shared
// memory: pull, collide, store straight to global memory (plus, next to a
// periodic end or a wall, the copies and ghost values it supplies), wall
// moments.
template <int Q, typename S, typename C, typename TB>
__device__ __forceinline__ void ws_update_cell_tb(const WsLattice<S>& L, const Consts<C>& k, const S* in,
                                                  const TB& tb, int i, int j, int r, int cc, int gcols) {
    using G = TileGeom<Q, S>;
    constexpr int H = Lat<Q>::H;
    // the cell's arithmetic carries the storage scale (values as stored)
    constexpr int SC = Store<S>::SCALE;
    Cell<Q, C> c;
    pull_cell<Q, C, SC>(
        [&](int al, int dr, int dc) -> C {
            return C(Store<S>::ldsr(in + G::off(al) + (r + G::row0(al) + dr) * G::width(al) + cc +
                                    G::col0(al) + dc));
        },
        tb, k, c);
    S* dst = L.dst + (long long)(i + H) * L.ld + j + GC;
    const int dw = wrap_offset(j, L.n2);
    const int pl = (int)L.plane;   // Q planes < 2^31 values (checked at creation)
    collide_emit<Q, C, SC>(tb, c, k, [&](int al, C v) {
        StStream<S>::str(dst + al * pl, v);
        if (dw != 0) StStream<S>::str(dst + (al * pl + dw), v);
    });
    if (EdgeFill<Q, S>::needed(i, L.n1, L.n2)) {
        const EdgeFill<Q, S> ef{L.dst, (const typename Store<S>::C*)L.ghost, L.plane, L.ld, L.n1, L.n2, L.bc_lo, L.bc_hi,
                                C(L.U0_lo), C(L.U0_hi), L.n2 < 2 * GC, gcols};
        ef.fill_inline(i, j, dst, L.plane, c.rho, c.Ut2);
    }
    if (i < H) {
        const int idx = i * L.n2 + j;
        ((C*)L.wall_rho)[idx] = c.rho;
        ((C*)L.wall_ut2)[idx] = c.Ut2;
    }
    if (i >= L.n1 - H) {
        const int idx = (H + (L.n1 - 1 - i)) * L.n2 + j;
        ((C*)L.wall_rho)[idx] = c.rho;
        ((C*)L.wall_ut2)[idx] = c.Ut2;
    }
}

// Planar and polar grids: the row's table block staged with the tile.
template <int Q, typename S, typename C>
__device__ __forceinline__ void ws_update_cell(const WsLattice<S>& L, const Consts<C>& k, const S* in,
                                               const C* tab_rows, int i0, int j0, int r, int cc) {
    const int i = i0 + r, j = j0 + cc;
    if (i >= L.n1 || j >= L.n2) return;
    ws_update_cell_tb<Q, S, C>(L, k, in, RowTab<Q, C>{tab_rows + r * Tab<Q>::S}, i, j, r, cc, 1);
}

// General grids: the cell's own table planes, read from global memory (one
// coalesced plane read per entry per warp), the state from the staged tile.
template <int Q, typename S, typename C>
__device__ __forceinline__ void ws_update_cell_gen(const WsLattice<S>& L, const Consts<C>& k, const S* in,
                                                   const C* tab, int i0, int j0, int r, int cc) {
    const int i = i0 + r, j = j0 + cc;
    if (i >= L.n1 || j >= L.n2) return;
    ws_update_cell_tb<Q, S, C>(L, k, in, TabOf<Q, C, true>::at(tab, i, j, L.n1, L.n2), i, j, r, cc, L.n2);
}

// Issue the TMA boxes of tile (i0, j0) from the 8 load maps of the source
// buffer, plus the tile's table rows, on barrier bar.
template <int Q, typename S, typename C, int TRO = 0>
__device__ __forceinline__ void ws_issue(const CUtensorMap* ld8, int i0, int j0, int n1, const C* tab,
                                         unsigned char* sm_in, unsigned char* sm_tab, uint64_t* bar) {
    using G = TileGeom<Q, S, TRO>;
    constexpr int H = Lat<Q>::H;
    const int nrows = n1 - i0 < G::TR ? n1 - i0 : G::TR;
    uint32_t bytes = tab ? (uint32_t)nrows * Tab<Q>::S * 4 : 0u;   // no rows: per-cell tables
#pragma unroll
    for (int al = 0; al < Q; ++al) bytes += G::rows(al) * G::width(al) * (int)sizeof(S);
    mbar_expect(bar, bytes);
    S* in = (S*)sm_in;
#pragma unroll
    for (int al = 0; al < Q; ++al)
        tma_load3(in + G::off(al), &ld8[G::shape(al)], j0 + GC - G::col0(al), i0 + H - G::row0(al), al, bar);
    if (tab) bulk_load(sm_tab, tab + (size_t)i0 * Tab<Q>::S, (uint32_t)nrows * Tab<Q>::S * 4, bar);
}

// The pipelined loop shared by the single-lattice and the batched updates
// and the residual: the CTA's t-th tile is tile_of(blockIdx.x + t gridDim.x, t)
// (every thread asks for t = 0, 1, 2, ... in order); tile_of fills (load
// maps, table, lat.n1, i0, j0) of a tile, and every
// consumer thread then runs cell(tile, staged boxes, staged table rows, r, cc)
// for its cell (r, cc) of the tile.  The producer warp re-fills a stage once
// all consumer warps released it; waits are bounded and a time-out records
// an error, stops the other warps at their next wait, and lets the loads in
// flight land before the CTA exits.  Every thread returns (the producer warp
// first), so a caller may follow with CTA-wide work.
//
// PUBLISH: the producer alone calls tile_of and stores the tile it returns in
// the stage's shared-memory slot before it issues the loads (the arrive that
// starts the stage's transaction count releases that store; the consumers'
// wait on the full barrier acquires it), and the consumers read the tile from
// there -- for tiles whose description sits in global memory (batches),
// which every consumer would otherwise fetch, with its latency, at every tile.
template <int Q, typename S, typename C, bool PUBLISH = false, int CPT = 1, int TRO = 0, typename TileOf,
          typename CellFn>
__device__ __forceinline__ void ws_pipeline(int ntiles, int* err, TileOf&& tile_of, CellFn&& cell) {
    using G = TileGeom<Q, S, TRO>;
    using P = PipeGeom<Q, S, CPT, TRO>;
    using Tile = decltype(tile_of(0, 0));
    static_assert(sizeof(Tile) <= P::TILE_SLOT, "tile descriptor exceeds its shared-memory slot");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* const smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t* const full = (uint64_t*)(smem + P::STAGES * P::STAGE_BYTES);
    uint64_t* const empty = full + P::STAGES;
    volatile int* const s_abort = (volatile int*)(empty + P::STAGES);
    Tile* const slots = (Tile*)(smem + P::STAGES * P::STAGE_BYTES + 2 * P::STAGES * 8 + 16);
    auto stage_in = [&](int st) { return smem + st * P::STAGE_BYTES; };
    auto stage_tab = [&](int st) { return smem + st * P::STAGE_BYTES + P::IN_BYTES; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int st = 0; st < P::STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], P::CONSUMERS);
        }
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == P::CONSUMERS) {  // producer
        if (lane == 0) {
            int it = 0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
                const int st = it % P::STAGES;
                if (it >= P::STAGES && !mbar_wait(&empty[st], (it / P::STAGES - 1) & 1)) {
                    *s_abort = 1;
                    atomicExch(err, 1);
                    break;
                }
                if (*s_abort) break;
                const Tile t = tile_of(tile, it);
                if (PUBLISH) slots[st] = t;
                ws_issue<Q, S, C, TRO>(t.ld8, t.i0, t.j0, t.lat.n1, t.tab, stage_in(st), stage_tab(st),
                                       &full[st]);
            }
            // the loads of the last issued tiles must land before the CTA exits
            for (int t = it > P::STAGES ? it - P::STAGES : 0; t < it; ++t)
                mbar_wait(&full[t % P::STAGES], (t / P::STAGES) & 1);
        }
        return;
    }

    // the consumer's cell (CPT = 2: cells cc and cc + 1, cc even)
    const int r = tid / (G::TJ / CPT), cc = (tid % (G::TJ / CPT)) * CPT;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int st = it % P::STAGES;
        if (!mbar_wait(&full[st], (it / P::STAGES) & 1)) {
            *s_abort = 1;
            atomicExch(err, 1);
            break;
        }
        if (*s_abort) break;
        if (PUBLISH) {
            const Tile t = slots[st];
            cell(t, (const S*)stage_in(st), (const C*)stage_tab(st), r, cc);
        } else {
            const Tile t = tile_of(tile, it);
            cell(t, (const S*)stage_in(st), (const C*)stage_tab(st), r, cc);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
    }
}

template <int Q, typename S, typename C>
struct WsTile {
    const CUtensorMap* ld8;
    const C* tab;
    WsLattice<S> lat;
    Consts<C> k;
    int i0, j0;
};

// The update of the consumer's cell of a WsTile.
template <int Q, typename S, typename C>
struct WsUpdate {
    __device__ __forceinline__ void operator()(const WsTile<Q, S, C>& t, const S* in, const C* tab, int r,
                                               int cc) const {
        ws_update_cell<Q, S, C>(t.lat, t.k, in, tab, t.i0, t.j0, r, cc);
    }
};

// The order in which a CTA walks the tiles of one lattice: tile
// blockIdx.x + t gridDim.x in row-major order (band-major: all CTAs work on a
// few neighbouring bands at a time, so every TMA box row is part of a long
// contiguous run that the other CTAs read at the same time).  Each thread
// steps its own copy from its t-th to its (t+1)-th tile without a division.
struct RowWalk {
    int band, col, cols, dband, dcol;
    __device__ __forceinline__ explicit RowWalk(int cols_) : cols(cols_) {
        band = (int)blockIdx.x / cols;
        col = (int)blockIdx.x - band * cols;
        dband = (int)gridDim.x / cols;
        dcol = (int)gridDim.x - dband * cols;
    }
    __device__ __forceinline__ void next() {
        band += dband;
        col += dcol;
        if (col >= cols) {
            col -= cols;
            ++band;
        }
    }
};

// The pipelined update of one lattice (PipeGeom): tile t of a CTA uses stage
// t mod STAGES.
template <int Q, typename S, typename C>
__global__ void __launch_bounds__((PipeGeom<Q, S>::NTHREADS), 1)
    k_fused_ws(const __grid_constant__ TmaMaps maps, const StepArgs a, int src) {
    using G = TileGeom<Q, S>;
    const int cols = (a.n2 + G::TJ - 1) / G::TJ;
    const int ntiles = ((a.n1 + G::TR - 1) / G::TR) * cols;
    const WsLattice<S> lat{(S*)a.dst, a.ghost, a.wall_rho, a.wall_ut2, a.plane, a.ld, a.n1, a.n2,
                           a.bc_lo, a.bc_hi, a.U0_lo, a.U0_hi};
    const Consts<C> k = Consts<C>::make(a.k);
    RowWalk w(cols);
    ws_pipeline<Q, S, C>(ntiles, a.err, [&](int, int t) {
        if (t > 0) w.next();
        return WsTile<Q, S, C>{maps.ld[src], (const C*)a.tab, lat, k, w.band * G::TR, w.col * G::TJ};
    }, WsUpdate<Q, S, C>{});
}

// Two neighbouring cells (i, j) and (i, j + 1), j even, of a tile staged in
// shared memory, computed together in the packed F2 arithmetic (the same
// update, each lane rounded as the scalar form): pull, collide, store both
// cells' values in one store per population, and per cell the periodic
// copies, ghost values and wall moments it supplies.
// Rows of the two-cells-per-thread update's tiles: 12 rows keep 12 consumer
// warps per SM at 128 registers without spills.  FP16 storage on the
// 1024 x 4096 annulus, per launch: 8 rows 8 warps, latency-bound (45 %
// issue-active against the one-cell kernel's 63 %); 10 rows 125.0 us; 12
// rows 105.7 us (one cell per thread: 110.9 us, with 29 % more
// instructions); 14 rows 113.6 us (four pipeline stages instead of five);
// 16 rows spill at 96 registers (114.8 us), and held to 120 registers
// with __maxnreg__ its 544 threads cannot be launched.
constexpr int PAIR_TR = 12;

template <int Q, typename S>
__device__ __forceinline__ void ws_update_pair(const WsLattice<S>& L, const Consts<F2>& k, const S* in,
                                               const float* tab_rows, int i0, int j0, int r, int cc) {
    using G = TileGeom<Q, S, PAIR_TR>;
    constexpr int H = Lat<Q>::H;
    constexpr int SC = Store<S>::SCALE;
    const int i = i0 + r, j = j0 + cc;
    if (i >= L.n1 || j >= L.n2) return;
    const bool both = j + 1 < L.n2;
    const RowTab2<Q> tb{tab_rows + r * Tab<Q>::S};
    Cell<Q, F2> c;
    pull_cell<Q, F2, SC>(
        [&](int al, int dr, int dc) -> F2 {
            const S* p = in + G::off(al) + (r + G::row0(al) + dr) * G::width(al) + cc + G::col0(al) + dc;
            // cc and col0 are even: the pair is aligned when the shift is
            return F2(((G::col0(al) + dc) & 1) ? Ld2<S, false>::ld(p) : Ld2<S, true>::ld(p));
        },
        tb, k, c);
    S* dst = L.dst + (long long)(i + H) * L.ld + j + GC;
    const int dwa = wrap_offset(j, L.n2), dwb = both ? wrap_offset(j + 1, L.n2) : 0;
    const int pl = (int)L.plane;
    // the periodic copies stay predicated stores beside the main one: a
    // separate pass reading the stored values back for the cells within GC
    // of a row's ends ran 27 % slower (134.5 against 105.7 us per launch)
    collide_emit<Q, F2, SC>(tb, c, k, [&](int al, F2 v) {
        St2<S>::st(dst + al * pl, v, both);
        if (dwa != 0) __stcs(dst + (al * pl + dwa), S(v.v.x));
        if (dwb != 0) __stcs(dst + (al * pl + 1 + dwb), S(v.v.y));
    });
    if (EdgeFill<Q, S>::needed(i, L.n1, L.n2)) {
        const EdgeFill<Q, S> ef{L.dst, (const typename Store<S>::C*)L.ghost, L.plane, L.ld, L.n1, L.n2, L.bc_lo, L.bc_hi,
                                float(L.U0_lo), float(L.U0_hi), L.n2 < 2 * GC, 1};
        ef.fill(i, j, dst, L.plane, c.rho.v.x, c.Ut2.v.x);
        if (both) ef.fill(i, j + 1, dst + 1, L.plane, c.rho.v.y, c.Ut2.v.y);
    }
    if (i < H || i >= L.n1 - H) {
        const int row = i < H ? i : H + (L.n1 - 1 - i);
        float* wr = (float*)L.wall_rho + row * L.n2 + j;
        float* wu = (float*)L.wall_ut2 + row * L.n2 + j;
        wr[0] = c.rho.v.x;
        wu[0] = c.Ut2.v.x;
        if (both) {
            wr[1] = c.rho.v.y;
            wu[1] = c.Ut2.v.y;
        }
    }
}

template <int Q, typename S>
struct WsUpdatePair {
    __device__ __forceinline__ void operator()(const WsTile<Q, S, float>& t, const S* in, const float* tab,
                                               int r, int cc) const {
        const Consts<float>& f = t.k;
        const Consts<F2> k2{F2(f.rho0), F2(f.g1), F2(f.g2), F2(f.tau_inv), F2(f.omt), F2(f.pref)};
        ws_update_pair<Q, S>(t.lat, k2, in, tab, t.i0, t.j0, r, cc);
    }
};

// The pipelined update with two cells per consumer thread: the same tiles,
// stages and producer, half as many consumer warps, each thread computing a
// pair of neighbouring cells in packed arithmetic (shared row table, paired
// loads and stores).
template <int Q, typename S>
__global__ void __launch_bounds__((PipeGeom<Q, S, 2, PAIR_TR>::NTHREADS), 1)
    k_fused_ws2(const __grid_constant__ TmaMaps maps, const StepArgs a, int src) {
    using G = TileGeom<Q, S, PAIR_TR>;
    const int cols = (a.n2 + G::TJ - 1) / G::TJ;
    const int ntiles = ((a.n1 + G::TR - 1) / G::TR) * cols;
    const WsLattice<S> lat{(S*)a.dst, a.ghost, a.wall_rho, a.wall_ut2, a.plane, a.ld, a.n1, a.n2,
                           a.bc_lo, a.bc_hi, a.U0_lo, a.U0_hi};
    RowWalk w(cols);
    ws_pipeline<Q, S, float, false, 2, PAIR_TR>(ntiles, a.err, [&](int, int t) {
        if (t > 0) w.next();
        return WsTile<Q, S, float>{maps.ld12[src], (const float*)a.tab, lat, Consts<float>::make(a.k),
                                   w.band * G::TR, w.col * G::TJ};
    }, WsUpdatePair<Q, S>{});
}

// General grids: the same pipeline, no table rows staged (the producer's
// table pointer is null); each consumer reads its cell's table planes.
template <int Q, typename S, typename C>
struct WsUpdateGen {
    const C* tab;
    __device__ __forceinline__ void operator()(const WsTile<Q, S, C>& t, const S* in, const C*, int r,
                                               int cc) const {
        ws_update_cell_gen<Q, S, C>(t.lat, t.k, in, tab, t.i0, t.j0, r, cc);
    }
};

template <int Q, typename S, typename C>
__global__ void __launch_bounds__((PipeGeom<Q, S>::NTHREADS), 1)
    k_fused_ws_gen(const __grid_constant__ TmaMaps maps, const StepArgs a, int src) {
    using G = TileGeom<Q, S>;
    const int cols = (a.n2 + G::TJ - 1) / G::TJ;
    const int ntiles = ((a.n1 + G::TR - 1) / G::TR) * cols;
    const WsLattice<S> lat{(S*)a.dst, a.ghost, a.wall_rho, a.wall_ut2, a.plane, a.ld, a.n1, a.n2,
                           a.bc_lo, a.bc_hi, a.U0_lo, a.U0_hi};
    const Consts<C> k = Consts<C>::make(a.k);
    RowWalk w(cols);
    ws_pipeline<Q, S, C>(ntiles, a.err, [&](int, int t) {
        if (t > 0) w.next();
        return WsTile<Q, S, C>{maps.ld[src], nullptr, lat, k, w.band * G::TR, w.col * G::TJ};
    }, WsUpdateGen<Q, S, C>{(const C*)a.tab});
}

// The pipelined update of a batch: work item e = (lattice, i0, j0) over all
// lattices' 8 x 64 tiles; maps holds each lattice's 2 x 8 load maps in global
// memory (written before the launch; acquired for the tensor-map proxy
// before use).
template <int Q, typename S, typename C>
__global__ void __launch_bounds__((PipeGeom<Q, S>::NTHREADS), 1)
    k_batch_ws(const BatchGrid* __restrict__ grids, const CUtensorMap* __restrict__ maps,
               const int4* __restrict__ work, int nwork, int parity, int* err) {
    const CUtensorMap* fenced = nullptr;  // producer: maps acquired last
    ws_pipeline<Q, S, C, true>(nwork, err, [&](int e, int) {
        const int4 w = work[e];
        const BatchGrid& g = grids[w.x];
        const int src = g.parity ^ parity;
        const CUtensorMap* ld8 = maps + ((size_t)w.x * 2 + src) * 8;
        if (ld8 != fenced && (threadIdx.x & 31) == 0 && threadIdx.x / 32 == PipeGeom<Q, S>::CONSUMERS) {
            for (int q = 0; q < 8; ++q)
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(ld8 + q)
                             : "memory");
            fenced = ld8;
        }
        const WsLattice<S> lat{(S*)g.phys[src ^ 1], g.ghost, g.wall_rho, g.wall_ut2, g.plane, g.ld,
                               g.n1, g.n2, g.bc_lo, g.bc_hi, g.U0_lo, g.U0_hi};
        return WsTile<Q, S, C>{ld8, (const C*)g.tab, lat, Consts<C>::make(g.k), w.y, w.z};
    }, WsUpdate<Q, S, C>{});
}

// Progress between the CTAs of a multi-step run (k_fused_ws_run).  Each CTA
// publishes, tagged with the launch's epoch, the run index of its oldest
// tile not yet complete (release at GPU scope: the consumers' stores,
// acquired by the producer through the stage's empty barrier, come with
// it); tiles are handed out in run order, so every tile below the minimum
// over the CTAs is complete.  A tile of step s > 0 in band b reads rows of
// bands b - 1 .. b + 1 of step s - 1 (the pull reaches |c^1| <= 3 rows,
// fewer than a band's; the periodic ghost columns and wall ghost rows a band
// writes serve its own rows) and overwrites rows those bands' tiles read: it
// waits until every tile of step s - 1 up to band b + 1 is complete, about a
// step behind the tiles in flight, so the last known minimum normally
// suffices.  Before it waits for real, the producer lets its consumers
// finish every tile it issued and publishes that, so the CTA holding the
// oldest incomplete tile always has its inputs: with every CTA resident (a
// cooperative launch) the run cannot deadlock.  Waits are bounded (error
// code 2).
struct RunSync {
    unsigned long long* prog;
    unsigned epoch;
    int per_step, cols, nbands, period;
    unsigned known;          // the producer's last minimum over the CTAs
    unsigned last;           // the CTA's last published value (published values only grow)
    volatile int* abort;     // the CTA's stop flag (a consumer's wait gave up)

    __device__ void publish(unsigned p) {
        if (p <= last) return;
        last = p;
        const unsigned long long v = ((unsigned long long)epoch << 32) | p;
        asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(prog + blockIdx.x), "l"(v) : "memory");
    }
    __device__ unsigned scan() const {
        unsigned m = 0xffffffffu;
        for (int c = 0; c < (int)gridDim.x; ++c) {
            unsigned long long v;
            asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(prog + c) : "memory");
            const unsigned p = (unsigned)(v >> 32) == epoch ? (unsigned)v : 0u;
            m = p < m ? p : m;
        }
        // acquire what the CTAs released; the TMA loads that follow read it
        // through the async proxy
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        asm volatile("fence.proxy.async.global;" ::: "memory");
        return m;
    }
    // iteration `it` of the CTA's tiles, run index `oldest` of its oldest incomplete tile
    __device__ void consumed(int it, unsigned oldest) {
        if (it % period == 0) publish(oldest);
    }
    template <typename D>
    __device__ bool ready(unsigned e, D&& drain) {
        const int s = (int)(e / (unsigned)per_step);
        if (s == 0) return true;
        const int band = (int)(e - (unsigned)s * per_step) / cols;
        const unsigned need = (unsigned)(s - 1) * per_step + (unsigned)min(band + 2, nbands) * cols;
        if (known >= need) return true;
        known = scan();
        if (known >= need) return true;
        if (!drain()) return false;
        publish(e);
        for (int k = 0; k < (1 << 20) && !*abort; ++k) {
            __nanosleep(256);
            known = scan();
            if (known >= need) return true;
        }
        return false;
    }
    template <typename D>
    __device__ void finish(D&& drain) {
        if (drain()) publish(0xffffffffu);
    }
};

// A tile of a multi-step run as the stage's slot carries it: the step's
// parity, the tile's origin, and stop (no tile: the run is over).
struct RunTile {
    int p, i0, j0, stop;
};

// nsteps time steps of the pipelined update in one launch.  The tiles of
// steps 0, 1, ..., nsteps - 1 form one sequence (step by step, band-major
// within a step); each CTA's producer takes the next one from a counter in
// global memory (prog[gridDim.x], zeroed before the launch), so that the
// CTAs keep to neighbouring tiles as in a single-step launch, and the first
// bands of a step are updated while the last bands of the step before are
// still in flight: a launch gap, ramp-up and tail once per run instead of
// once per step.  Step s reads buffer src ^ (s & 1) and writes the other;
// CPT as in ws_pipeline; period: tiles between two progress publications.
// 16-bit storage (issue-bound) gains from it; FP32 storage (HBM-bound) ran
// slower than a launch per step however the tiles were shared out.
template <int Q, typename S, typename C, int CPT>
__global__ void __launch_bounds__((PipeGeom<Q, S, CPT, CPT == 2 ? PAIR_TR : 0>::NTHREADS), 1)
    k_fused_ws_run(const __grid_constant__ TmaMaps maps, const StepArgs a, int src, int nsteps,
                   unsigned long long* prog, unsigned epoch, int period) {
    constexpr int TRO = CPT == 2 ? PAIR_TR : 0;
    using G = TileGeom<Q, S, TRO>;
    using P = PipeGeom<Q, S, CPT, TRO>;
    using Update = typename std::conditional<CPT == 2, WsUpdatePair<Q, S>, WsUpdate<Q, S, C>>::type;
    const int cols = (a.n2 + G::TJ - 1) / G::TJ;
    const int nbands = (a.n1 + G::TR - 1) / G::TR;
    const int per_step = nbands * cols;
    const unsigned ntiles = (unsigned)per_step * (unsigned)nsteps;
    unsigned long long* const next = prog + gridDim.x;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* const smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t* const full = (uint64_t*)(smem + P::STAGES * P::STAGE_BYTES);
    uint64_t* const empty = full + P::STAGES;
    volatile int* const s_abort = (volatile int*)(empty + P::STAGES);
    volatile RunTile* const slots = (volatile RunTile*)(smem + P::STAGES * P::STAGE_BYTES + 2 * P::STAGES * 8 + 16);
    auto stage_in = [&](int st) { return smem + st * P::STAGE_BYTES; };
    auto stage_tab = [&](int st) { return smem + st * P::STAGE_BYTES + P::IN_BYTES; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int st = 0; st < P::STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], P::CONSUMERS);
        }
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == P::CONSUMERS) {  // producer
        if (lane == 0) {
            RunSync rs{prog, epoch, per_step, cols, nbands, period, 0u, 0u, s_abort};
            bool stopped = false;
            unsigned taken[P::STAGES];   // run index of the tile of each stage
            int it = 0;
            auto drain = [&]() {
                for (int t = it > P::STAGES ? it - P::STAGES : 0; t < it; ++t)
                    if (!mbar_wait(&empty[t % P::STAGES], (t / P::STAGES) & 1)) return false;
                return true;
            };
            unsigned e = (unsigned)atomicAdd(next, 1ull);
            for (;; ++it) {
                const int st = it % P::STAGES;
                if (it >= P::STAGES) {
                    if (!mbar_wait(&empty[st], (it / P::STAGES - 1) & 1)) {
                        *s_abort = 1;
                        atomicExch(a.err, 1);
                        break;
                    }
                    rs.consumed(it, taken[(it - P::STAGES + 1) % P::STAGES]);
                }
                if (*s_abort) break;
                if (e >= ntiles) {   // the run is over: stop the consumers
                    slots[st].stop = 1;
                    mbar_arrive(&full[st]);
                    stopped = true;
                    break;
                }
                if (!rs.ready(e, drain)) {
                    *s_abort = 1;
                    atomicExch(a.err, 2);
                    break;
                }
                // the next tile is taken now, its latency hidden behind this one's loads
                const unsigned e_next = (unsigned)atomicAdd(next, 1ull);
                const int s = (int)(e / (unsigned)per_step), t = (int)(e - (unsigned)s * per_step);
                const int band = t / cols, col = t - band * cols, par = s & 1;
                slots[st].p = par;
                slots[st].i0 = band * G::TR;
                slots[st].j0 = col * G::TJ;
                slots[st].stop = 0;
                taken[st] = e;
                ws_issue<Q, S, C, TRO>(CPT == 2 ? maps.ld12[src ^ par] : maps.ld[src ^ par], band * G::TR,
                                       col * G::TJ, a.n1, (const C*)a.tab, stage_in(st), stage_tab(st), &full[st]);
                e = e_next;
            }
            // the loads of the last issued tiles must land before the CTA exits
            // (after a stop, whose arrive completed one more phase of its
            // stage, the tile issued STAGES iterations before it is known to
            // have landed: its stage was released)
            const int first = it > P::STAGES ? it - P::STAGES + (stopped ? 1 : 0) : 0;
            for (int t = first; t < it; ++t) mbar_wait(&full[t % P::STAGES], (t / P::STAGES) & 1);
            if (!*s_abort) rs.finish(drain);
        }
        return;
    }

    // consumers: the tiles the producer hands over, until the stop (a wait
    // for the next tile may include the producer's wait for the step before:
    // a longer bound than the single-step pipeline's)
    WsLattice<S> lat{(S*)a.dst, a.ghost, a.wall_rho, a.wall_ut2, a.plane, a.ld, a.n1, a.n2,
                     a.bc_lo, a.bc_hi, a.U0_lo, a.U0_hi};
    const Consts<C> k = Consts<C>::make(a.k);
    const int r = tid / (G::TJ / CPT), cc = (tid % (G::TJ / CPT)) * CPT;
    for (int it = 0;; ++it) {
        const int st = it % P::STAGES;
        if (!mbar_wait_n(&full[st], (it / P::STAGES) & 1, 1 << 22)) {
            *s_abort = 1;
            atomicExch(a.err, 1);
            break;
        }
        if (*s_abort || slots[st].stop) break;
        const int par = slots[st].p;
        lat.dst = par ? (S*)a.src : (S*)a.dst;   // written by even / odd steps
        const WsTile<Q, S, C> tile{nullptr, (const C*)a.tab, lat, k, slots[st].i0, slots[st].j0};
        Update{}(tile, (const S*)stage_in(st), (const C*)stage_tab(st), r, cc);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
    }
}

// A tile of the residual: what the producer needs (maps, table, n1, origin).
template <typename C>
struct ResTile {
    const CUtensorMap* ld8;
    const C* tab;
    struct {
        int n1;
    } lat;
    int i0, j0;
};

// The residual and conservation sums of clbm_residual over tiles staged by
// the same pipeline as the update: each consumer thread pulls its cell from
// shared memory, forms rho, U, F and Ut exactly as the update does (Eqs. 7-18,
// lagged force), and accumulates the cell's residual terms (ResAcc, a fixed
// order per thread: the tiles of a CTA are fixed); the CTA then reduces its
// threads in a fixed tree into one partial.  The loads stream through three
// stages instead of waiting cell by cell, so the pass runs near the
// bandwidth of one read of the state.
template <int Q, typename S, typename C>
__global__ void __launch_bounds__((PipeGeom<Q, S>::NTHREADS), 1)
    k_residual_ws(const __grid_constant__ TmaMaps maps, const MomArgs a, int src) {
    using G = TileGeom<Q, S>;
    const int cols = (a.n2 + G::TJ - 1) / G::TJ;
    const int ntiles = ((a.n1 + G::TR - 1) / G::TR) * cols;
    const Consts<C> k = Consts<C>::make(a.k);
    const size_t nc = (size_t)a.n1 * a.n2;
    C* const prev = (C*)a.ut_prev;
    const bool have_prev = a.have_prev != 0;
    ResAcc<C> acc;
    RowWalk w(cols);
    ws_pipeline<Q, S, C>(ntiles, a.err, [&](int, int t) {
        if (t > 0) w.next();
        return ResTile<C>{maps.ld[src], (const C*)a.tab, {a.n1}, w.band * G::TR, w.col * G::TJ};
    }, [&](const ResTile<C>& t, const S* in, const C* tab, int r, int cc) {
        const int i = t.i0 + r, j = t.j0 + cc;
        if (i >= a.n1 || j >= a.n2) return;
        const size_t m = (size_t)i * a.n2 + j;
        // the snapshot comes from global memory: load it first, so that its
        // latency hides behind the pull and the moments
        const C p1 = have_prev ? prev[m] : C(0), p2 = have_prev ? prev[nc + m] : C(0);
        const RowTab<Q, C> tb{tab + r * Tab<Q>::S};
        Cell<Q, C> c;
        pull_cell<Q, C>(
            [&](int al, int dr, int dc) -> C {
                return C(Store<S>::lds(in + G::off(al) + (r + G::row0(al) + dr) * G::width(al) + cc +
                                       G::col0(al) + dc));
            },
            tb, k, c);
        collide_emit<Q, C>(tb, c, k, [](int, C) {});
        acc.add(residual_terms<Q, C>(c, tb, p1, p2, have_prev));
        prev[m] = c.Ut1;
        prev[nc + m] = c.Ut2;
    });
    double v[NRED];
    acc.out(v);
    block_partial<PipeGeom<Q, S>::NTHREADS>(v, a.partial + (size_t)blockIdx.x * NRED);
}

}  // namespace

template <int Q, typename S>
static int run_ws(const TmaMaps& maps, const StepArgs& a, int src, int nsm, cudaStream_t s) {
    using G = TileGeom<Q, S>;
    using P = PipeGeom<Q, S>;
    using C = typename Store<S>::C;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_fused_ws<Q, S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 P::SMEM) != cudaSuccess)
            return -1;
        attr_set[dev] = true;
    }
    const int tiles = ((a.n1 + G::TR - 1) / G::TR) * ((a.n2 + G::TJ - 1) / G::TJ);
    const int grid = tiles < nsm ? tiles : nsm;
    k_fused_ws<Q, S, C><<<grid, P::NTHREADS, P::SMEM, s>>>(maps, a, src);
    return 0;
}

template <int Q, typename S>
static int run_ws2(const TmaMaps& maps, const StepArgs& a, int src, int nsm, cudaStream_t s) {
    using G = TileGeom<Q, S, PAIR_TR>;
    using P = PipeGeom<Q, S, 2, PAIR_TR>;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_fused_ws2<Q, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, P::SMEM) !=
            cudaSuccess)
            return -1;
        attr_set[dev] = true;
    }
    const int tiles = ((a.n1 + G::TR - 1) / G::TR) * ((a.n2 + G::TJ - 1) / G::TJ);
    const int grid = tiles < nsm ? tiles : nsm;
    k_fused_ws2<Q, S><<<grid, P::NTHREADS, P::SMEM, s>>>(maps, a, src);
    return 0;
}

template <int Q, typename S, int CPT>
static cudaError_t run_ws_run(const TmaMaps& maps, const StepArgs& a, int src, int nsm, int nsteps,
                              unsigned long long* prog, unsigned epoch, cudaStream_t s) {
    constexpr int TRO = CPT == 2 ? PAIR_TR : 0;
    using G = TileGeom<Q, S, TRO>;
    using P = PipeGeom<Q, S, CPT, TRO>;
    using C = typename Store<S>::C;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(k_fused_ws_run<Q, S, C, CPT>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, P::SMEM);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    const int tiles = ((a.n1 + G::TR - 1) / G::TR) * ((a.n2 + G::TJ - 1) / G::TJ);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tiles < nsm ? tiles : nsm);
    cfg.blockDim = dim3(P::NTHREADS);
    cfg.dynamicSmemBytes = P::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // every CTA resident: the run orders its steps itself
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // publish progress every `period` tiles: as rarely as the run allows
    // (each is a release at GPU scope) while the slowest CTA's published
    // tile stays more than a step's worth of tiles minus two bands behind
    // the tiles in flight, so that waits are met without draining
    const int cols = (a.n2 + G::TJ - 1) / G::TJ, grid = tiles < nsm ? tiles : nsm;
    int period = 1;
    while (period < 64 && (4 * period + P::STAGES + 2) * grid <= tiles - 2 * cols) period *= 2;
    // the run's tile counter, after the grid's progress words
    const cudaError_t e = cudaMemsetAsync(prog + grid, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, k_fused_ws_run<Q, S, C, CPT>, maps, a, src, nsteps, prog, epoch, period);
}

template <int Q, typename S>
static cudaError_t run_mode_run(int mode, const TmaMaps& maps, const StepArgs& a, int src, int nsm, int nsteps,
                                unsigned long long* prog, unsigned epoch, cudaStream_t s) {
    return mode == 2 ? run_ws_run<Q, S, 2>(maps, a, src, nsm, nsteps, prog, epoch, s)
                     : run_ws_run<Q, S, 1>(maps, a, src, nsm, nsteps, prog, epoch, s);
}

template <int Q, typename S>
static int run_batch_ws(const BatchGrid* grids, const void* maps, const int4* work, int nwork, int parity,
                        int nsm, int* err, cudaStream_t s) {
    using P = PipeGeom<Q, S>;
    using C = typename Store<S>::C;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_batch_ws<Q, S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 P::SMEM) != cudaSuccess)
            return -1;
        attr_set[dev] = true;
    }
    const int grid = nwork < nsm ? nwork : nsm;
    k_batch_ws<Q, S, C><<<grid, P::NTHREADS, P::SMEM, s>>>(grids, (const CUtensorMap*)maps, work, nwork,
                                                          parity, err);
    return 0;
}

template <int Q, typename S>
static int run_residual_ws(const TmaMaps& maps, const MomArgs& m, int src, int nsm, cudaStream_t s) {
    using G = TileGeom<Q, S>;
    using P = PipeGeom<Q, S>;
    using C = typename Store<S>::C;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_residual_ws<Q, S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 P::SMEM) != cudaSuccess)
            return -1;
        attr_set[dev] = true;
    }
    const int tiles = ((m.n1 + G::TR - 1) / G::TR) * ((m.n2 + G::TJ - 1) / G::TJ);
    const int grid = tiles < nsm ? tiles : nsm;
    k_residual_ws<Q, S, C><<<grid, P::NTHREADS, P::SMEM, s>>>(maps, m, src);
    return grid;
}

int launch_residual_tma(int Q, int prec, const TmaMaps& maps, const MomArgs& m, int src, int nsm,
                        cudaStream_t s) {
    if (Q == 9) {
        switch (prec) {
            case 1: return run_residual_ws<9, float>(maps, m, src, nsm, s);
            case 2: return run_residual_ws<9, __half>(maps, m, src, nsm, s);
            case 3: return run_residual_ws<9, __nv_bfloat16>(maps, m, src, nsm, s);
            default: return -1;
        }
    }
    switch (prec) {
        case 1: return run_residual_ws<21, float>(maps, m, src, nsm, s);
        case 2: return run_residual_ws<21, __half>(maps, m, src, nsm, s);
        case 3: return run_residual_ws<21, __nv_bfloat16>(maps, m, src, nsm, s);
        default: return -1;
    }
}

int launch_batch_ws(int Q, int prec, const BatchGrid* grids, const void* maps, const int4* work, int nwork,
                    int parity, int nsm, int* err, cudaStream_t s) {
    if (nwork <= 0) return 0;
    if (Q == 9) {
        switch (prec) {
            case 1: return run_batch_ws<9, float>(grids, maps, work, nwork, parity, nsm, err, s);
            case 2: return run_batch_ws<9, __half>(grids, maps, work, nwork, parity, nsm, err, s);
            case 3: return run_batch_ws<9, __nv_bfloat16>(grids, maps, work, nwork, parity, nsm, err, s);
            default: return -1;
        }
    }
    switch (prec) {
        case 1: return run_batch_ws<21, float>(grids, maps, work, nwork, parity, nsm, err, s);
        case 2: return run_batch_ws<21, __half>(grids, maps, work, nwork, parity, nsm, err, s);
        case 3: return run_batch_ws<21, __nv_bfloat16>(grids, maps, work, nwork, parity, nsm, err, s);
        default: return -1;
    }
}

size_t tma_load_maps(const TmaMaps* m, void* out) {
    const size_t bytes = sizeof(m->ld);
    if (out) memcpy(out, m->ld, bytes);
    return bytes;
}

template <int Q, typename S>
static int run_tma(const TmaMaps& maps, const StepArgs& a, int src, int nsm, cudaStream_t s) {
    using G = TileGeom<Q, S>;
    using C = typename Store<S>::C;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_fused_tma<Q, S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 G::SMEM) != cudaSuccess)
            return -1;
        attr_set[dev] = true;
    }
    const int tiles = ((a.n1 + G::TR - 1) / G::TR) * ((a.n2 + G::TJ - 1) / G::TJ);
    const int grid = tiles < nsm ? tiles : nsm;
    k_fused_tma<Q, S, C><<<grid, G::NT, G::SMEM, s>>>(maps, a, src);
    return 0;
}

template <int Q, typename S>
static int run_ws_gen(const TmaMaps& maps, const StepArgs& a, int src, int nsm, cudaStream_t s) {
    using G = TileGeom<Q, S>;
    using P = PipeGeom<Q, S>;
    using C = typename Store<S>::C;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_fused_ws_gen<Q, S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 P::SMEM) != cudaSuccess)
            return -1;
        attr_set[dev] = true;
    }
    const int tiles = ((a.n1 + G::TR - 1) / G::TR) * ((a.n2 + G::TJ - 1) / G::TJ);
    const int grid = tiles < nsm ? tiles : nsm;
    k_fused_ws_gen<Q, S, C><<<grid, P::NTHREADS, P::SMEM, s>>>(maps, a, src);
    return 0;
}

int launch_step_tma_general(int Q, int prec, const TmaMaps& maps, const StepArgs& a, int src, int nsm,
                            cudaStream_t s) {
    if (Q == 9) {
        switch (prec) {
            case 1: return run_ws_gen<9, float>(maps, a, src, nsm, s);
            case 2: return run_ws_gen<9, __half>(maps, a, src, nsm, s);
            case 3: return run_ws_gen<9, __nv_bfloat16>(maps, a, src, nsm, s);
            default: return -1;
        }
    }
    switch (prec) {
        case 1: return run_ws_gen<21, float>(maps, a, src, nsm, s);
        case 2: return run_ws_gen<21, __half>(maps, a, src, nsm, s);
        case 3: return run_ws_gen<21, __nv_bfloat16>(maps, a, src, nsm, s);
        default: return -1;
    }
}

template <int Q, typename S>
static int run_mode(int mode, const TmaMaps& maps, const StepArgs& a, int src, int nsm, cudaStream_t s) {
    return mode == 0 ? run_tma<Q, S>(maps, a, src, nsm, s)
         : mode == 1 ? run_ws<Q, S>(maps, a, src, nsm, s)
                     : run_ws2<Q, S>(maps, a, src, nsm, s);
}

// mode 0: TMA tiles with a shared output tile; 1: the pipelined update; 2:
// the pipelined update with two cells per consumer thread.
int launch_step_tma(int Q, int prec, const TmaMaps& maps, const StepArgs& a, int src, int nsm, int mode,
                    cudaStream_t s) {
    if (Q == 9) {
        switch (prec) {
            case 1: return run_mode<9, float>(mode, maps, a, src, nsm, s);
            case 2: return run_mode<9, __half>(mode, maps, a, src, nsm, s);
            case 3: return run_mode<9, __nv_bfloat16>(mode, maps, a, src, nsm, s);
            default: return -1;
        }
    }
    switch (prec) {
        case 1: return run_mode<21, float>(mode, maps, a, src, nsm, s);
        case 2: return run_mode<21, __half>(mode, maps, a, src, nsm, s);
        case 3: return run_mode<21, __nv_bfloat16>(mode, maps, a, src, nsm, s);
        default: return -1;
    }
}

// Tiles per time step of the pipelined update (mode 1 or 2) on an n1 x n2 grid.
int run_tiles(int Q, int mode, int n1, int n2) {
    const int tr = mode == 2 ? PAIR_TR : Q == 9 ? TileGeom<9, float>::TR : TileGeom<21, float>::TR;
    const int tj = TileGeom<21, float>::TJ;
    return ((n1 + tr - 1) / tr) * ((n2 + tj - 1) / tj);
}

cudaError_t launch_step_tma_run(int Q, int prec, const TmaMaps& maps, const StepArgs& a, int src, int nsm,
                                int mode, int nsteps, unsigned long long* prog, unsigned epoch,
                                cudaStream_t s) {
    if (Q == 9) {
        switch (prec) {
            case 1: return run_mode_run<9, float>(mode, maps, a, src, nsm, nsteps, prog, epoch, s);
            case 2: return run_mode_run<9, __half>(mode, maps, a, src, nsm, nsteps, prog, epoch, s);
            case 3: return run_mode_run<9, __nv_bfloat16>(mode, maps, a, src, nsm, nsteps, prog, epoch, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (prec) {
        case 1: return run_mode_run<21, float>(mode, maps, a, src, nsm, nsteps, prog, epoch, s);
        case 2: return run_mode_run<21, __half>(mode, maps, a, src, nsm, nsteps, prog, epoch, s);
        case 3: return run_mode_run<21, __nv_bfloat16>(mode, maps, a, src, nsm, nsteps, prog, epoch, s);
        default: return cudaErrorInvalidValue;
    }
}

// Encode the tensor maps of both state buffers (host).
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                              CUtensorMapFloatOOBfill);

template <int Q, typename S>
static int encode_maps(EncodeFn enc, TmaMaps* m, void* bufA, void* bufB, int n1, int n2, int ld,
                       CUtensorMapDataType dt) {
    using G = TileGeom<Q, S>;
    constexpr int H = Lat<Q>::H;
    const cuuint64_t es = sizeof(S);
    cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)(n1 + 2 * H), (cuuint64_t)Q};
    cuuint64_t strides[2] = {(cuuint64_t)ld * es, (cuuint64_t)(n1 + 2 * H) * ld * es};
    cuuint32_t estr[3] = {1, 1, 1};
    void* bases[2] = {bufA, bufB};
    for (int b = 0; b < 2; ++b) {
        for (int shape = 0; shape < 8; ++shape) {
            const int ac1 = shape / 2, has2 = shape & 1;
            cuuint32_t box[3] = {(cuuint32_t)(has2 ? G::TJ + 2 * G::HX : G::TJ), (cuuint32_t)(G::TR + ac1), 1};
            if (enc(&m->ld[b][shape], dt, 3, bases[b], dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return -1;
            using G12 = TileGeom<Q, S, PAIR_TR>;
            cuuint32_t box12[3] = {(cuuint32_t)(has2 ? G12::TJ + 2 * G12::HX : G12::TJ),
                                   (cuuint32_t)(G12::TR + ac1), 1};
            if (enc(&m->ld12[b][shape], dt, 3, bases[b], dims, strides, box12, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return -1;
        }
        // interior view for the tile store: origin at (row H, column GC), rows
        // cut at the last whole 16-byte chunk (a partial chunk would be
        // written whole, into the ghost columns)
        char* ib = (char*)bases[b] + ((size_t)H * ld + GC) * es;
        const int n2v = tma_store_cols<S>(n2);
        if (n2v < 1) return -1;
        cuuint64_t idims[3] = {(cuuint64_t)n2v, (cuuint64_t)n1, (cuuint64_t)Q};
        cuuint32_t obox[3] = {(cuuint32_t)G::TJ, (cuuint32_t)G::TR, (cuuint32_t)Q};
        if (enc(&m->st[b], dt, 3, ib, idims, strides, obox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return -1;
    }
    return 0;
}

int make_tma_maps(int Q, int prec, TmaMaps** out, void* bufA, void* bufB, int n1, int n2, int ld) {
    static EncodeFn enc = nullptr;
    if (!enc) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        enc = (EncodeFn)fn;
    }
    TmaMaps* m = new TmaMaps();
    int rc = -1;
    if (Q == 9) {
        if (prec == 1) rc = encode_maps<9, float>(enc, m, bufA, bufB, n1, n2, ld, CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
        else if (prec == 2) rc = encode_maps<9, __half>(enc, m, bufA, bufB, n1, n2, ld, CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
        else if (prec == 3) rc = encode_maps<9, __nv_bfloat16>(enc, m, bufA, bufB, n1, n2, ld, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    } else {
        if (prec == 1) rc = encode_maps<21, float>(enc, m, bufA, bufB, n1, n2, ld, CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
        else if (prec == 2) rc = encode_maps<21, __half>(enc, m, bufA, bufB, n1, n2, ld, CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
        else if (prec == 3) rc = encode_maps<21, __nv_bfloat16>(enc, m, bufA, bufB, n1, n2, ld, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    }
    if (rc != 0) {
        delete m;
        return -1;
    }
    *out = m;
    return 0;
}

void free_tma_maps(TmaMaps* m) { delete m; }

}  // namespace clbm
