// md_tile.cu -- one MD step of variant B (Sec. 3, Eqs. (4)-(8)) as one pass
// over tiles of lattice rows, plus a short follow-up.
//
// The particles are bucketed by the lattice row (y, z) of their cell at every
// re-ordering, and the active nodes (corners of the particles' cells) keep
// their node record in a compact array, row by row.  A block owns a tile of
// TILE_Y x TILE_Z lattice rows: the node rows and the particle buckets of
// those rows.  A particle in cell row (y, z) reads and feeds the nodes of the
// rows (y + oy, z + oz), oy, oz in {0, 1}, i.e. the tile's rows and one row
// above it in y and in z.  So a block
//   1. copies its tile's table (record and particle ranges, built once per
//      re-ordering by tile_table_kernel) and then the compact records of its
//      (TILE_Y + 1) x (TILE_Z + 1) rows into shared memory with bulk copies
//      (cp.async.bulk, the TMA engine; one copy per contiguous run of rows,
//      completion on an mbarrier), while each thread loads its particle;
//   2. runs the MD step of each of its particles from shared memory:
//      interpolation (Eq. (5)), friction and random force (Eq. (4)), velocity
//      Verlet with the force of the start of the step (Eq. (6)); each
//      transfer -delta_k Delta P (Eqs. (7), (8)) to a node of its own rows is
//      summed as a fixed-point integer in shared memory, one to the row above
//      the tile (owned by the next tile up in y or z) is added with an integer
//      atomic to an edge accumulator E in global memory;
//   3. publishes that its particles are done (a flag tagged with the MD step),
//      and writes its rows' new records, old value plus the sums, into the
//      second record buffer; a row at the tile's lower edge also takes the
//      edge accumulator filled by the tiles below, once their flags show them
//      done (they come earlier in the grid, so the wait is short and cannot
//      deadlock; it is bounded, and a row whose wait runs out is left to the
//      follow-up), and clears it.
// md_tile_finish_kernel then folds the edge accumulator of the rows at y = 0
// or z = 0 (their lower neighbours wrap to the far end of the grid) and of
// any row whose wait ran out, and spreads the listed particles with atomics:
// those that left their bucket's row since the re-ordering, or whose cell has
// a corner that is not active (they read the nodes from global memory).
// Every particle reads the records as they were at the start of the MD step
// (the old buffer), so all particles read the nodes before any transfer of
// the step is applied (the Jacobi order of Sec. 3).  A tile whose records
// exceed the shared memory reads them from global memory and adds its own
// rows' transfers with atomics into the new buffer (after copying its old
// records there).  Integer sums make every path give the same bits as the
// row gather and the all-atomic spreading.
#include "lbmd_ctx.h"
#include "particle_step.cuh"

namespace lbmd {

constexpr int TILE_Y = 4, TILE_Z = 4;
constexpr int TILE_THREADS = 256;
constexpr int TILE_WARPS = TILE_THREADS / 32;
constexpr int TILE_SR = (TILE_Y + 1) * (TILE_Z + 1);  // staged rows: the tile's and one above in y, z
constexpr int TILE_NO = TILE_Y * TILE_Z;              // the tile's rows (node rows and particle buckets)
constexpr int TILE_WMAX = 16;                         // active words per row: nx <= 512
constexpr int TILE_NSEG = 2 * (TILE_Z + 1);           // bulk copies: a z-line splits at most once (y wrap)
constexpr int TILE_SPIN = 1 << 20;                    // polls of a wait, at most (64 ns apart for flags)
static_assert(TILE_SR * TILE_WMAX <= 2 * TILE_THREADS, "two active words per thread at most");
static_assert(TILE_NSEG <= 32 && TILE_NO <= 32 && TILE_SR <= 32, "one warp builds a table");

// Shared-memory capacity of a tile (records staged, the tile's records summed).
template <typename T>
struct TileCap;
template <>
struct TileCap<float> {
    static constexpr int REC = 2816, ACC = 1792;
};
template <>
struct TileCap<double> {
    static constexpr int REC = 1408, ACC = 896;
};

// Shared-memory sums of the transfers to the owned records.  FP32: the x and
// y components in one 64-bit integer S = dy 2^32 + dx (the node record's own
// packing, so one 64-bit and one 32-bit atomic per transfer) and z apart;
// FP64: three 64-bit integers.  take() adds a record's sums to it.  The edge
// accumulator in global memory has the same layout per compact slot.
template <typename T>
struct TileAcc;
template <>
struct TileAcc<float> {
    __host__ __device__ static constexpr size_t bytes(int cap) { return (size_t)cap * 12; }
    __device__ static __forceinline__ void clear(unsigned char *base, int cap, int n, int tid, int nthreads) {
        unsigned long long *s = reinterpret_cast<unsigned long long *>(base);
        int *z = reinterpret_cast<int *>(base + (size_t)8 * cap);
        for (int k = tid; k < n; k += nthreads) {
            s[k] = 0ull;
            z[k] = 0;
        }
    }
    __device__ static __forceinline__ void add(unsigned char *base, int cap, int i, int32_t dx, int32_t dy,
                                               int32_t dz) {
        unsigned long long *s = reinterpret_cast<unsigned long long *>(base);
        int *z = reinterpret_cast<int *>(base + (size_t)8 * cap);
        atomicAdd(&s[i], (unsigned long long)((long long)dy * 4294967296LL + (long long)dx));
        atomicAdd(&z[i], dz);
    }
    __device__ static __forceinline__ void take(const unsigned char *base, int cap, int i, int4 &rec) {
        const unsigned long long *s = reinterpret_cast<const unsigned long long *>(base);
        const int *z = reinterpret_cast<const int *>(base + (size_t)8 * cap);
        const unsigned long long old = ((unsigned long long)(unsigned)rec.w << 32) | (unsigned)rec.z;
        const unsigned long long sum = old + s[i];
        rec.z = (int)(unsigned)sum;
        rec.w = (int)(unsigned)(sum >> 32);
        rec.y += z[i];
    }
    // the edge accumulator in global memory (cap records): read through L2,
    // added to rec, cleared
    __device__ static __forceinline__ void take_clear_global(unsigned char *base, int64_t cap, int64_t i,
                                                             int4 &rec) {
        unsigned long long *s = reinterpret_cast<unsigned long long *>(base);
        int *z = reinterpret_cast<int *>(base + (size_t)8 * cap);
        const unsigned long long S = __ldcg(&s[i]);
        const int dz = __ldcg(&z[i]);
        if (S == 0ull && dz == 0) return;
        const unsigned long long old = ((unsigned long long)(unsigned)rec.w << 32) | (unsigned)rec.z;
        const unsigned long long sum = old + S;
        rec.z = (int)(unsigned)sum;
        rec.w = (int)(unsigned)(sum >> 32);
        rec.y += dz;
        s[i] = 0ull;
        z[i] = 0;
    }
    // the same, added with atomics to a record other threads may update too
    __device__ static __forceinline__ void fold_atomic(unsigned char *base, int64_t cap, int64_t i, int4 *rec) {
        unsigned long long *s = reinterpret_cast<unsigned long long *>(base);
        int *z = reinterpret_cast<int *>(base + (size_t)8 * cap);
        const unsigned long long S = __ldcg(&s[i]);
        const int dz = __ldcg(&z[i]);
        if (S == 0ull && dz == 0) return;
        atomicAdd(reinterpret_cast<unsigned long long *>(&rec->z), S);
        atomicAdd(&rec->y, dz);
        s[i] = 0ull;
        z[i] = 0;
    }
};
template <>
struct TileAcc<double> {
    __host__ __device__ static constexpr size_t bytes(int cap) { return (size_t)cap * 24; }
    __device__ static __forceinline__ void clear(unsigned char *base, int, int n, int tid, int nthreads) {
        long long *s = reinterpret_cast<long long *>(base);
        for (int k = tid; k < 3 * n; k += nthreads) s[k] = 0;
    }
    __device__ static __forceinline__ void add(unsigned char *base, int, int i, long long dx, long long dy,
                                               long long dz) {
        unsigned long long *s = reinterpret_cast<unsigned long long *>(base) + 3 * (size_t)i;
        atomicAdd(s + 0, (unsigned long long)dx);
        atomicAdd(s + 1, (unsigned long long)dy);
        atomicAdd(s + 2, (unsigned long long)dz);
    }
    __device__ static __forceinline__ void take(const unsigned char *base, int, int i, L4 &rec) {
        const long long *s = reinterpret_cast<const long long *>(base) + 3 * (size_t)i;
        rec.y += s[0];
        rec.z += s[1];
        rec.w += s[2];
    }
    __device__ static __forceinline__ void take_clear_global(unsigned char *base, int64_t, int64_t i, L4 &rec) {
        long long *s = reinterpret_cast<long long *>(base) + 3 * (size_t)i;
        const long long d0 = __ldcg(s), d1 = __ldcg(s + 1), d2 = __ldcg(s + 2);
        if (d0 == 0 && d1 == 0 && d2 == 0) return;
        rec.y += d0;
        rec.z += d1;
        rec.w += d2;
        s[0] = s[1] = s[2] = 0;
    }
    __device__ static __forceinline__ void fold_atomic(unsigned char *base, int64_t, int64_t i, L4 *rec) {
        long long *s = reinterpret_cast<long long *>(base) + 3 * (size_t)i;
        const long long d0 = __ldcg(s), d1 = __ldcg(s + 1), d2 = __ldcg(s + 2);
        if (d0 == 0 && d1 == 0 && d2 == 0) return;
        atomicAdd(reinterpret_cast<unsigned long long *>(&rec->y), (unsigned long long)d0);
        atomicAdd(reinterpret_cast<unsigned long long *>(&rec->z), (unsigned long long)d1);
        atomicAdd(reinterpret_cast<unsigned long long *>(&rec->w), (unsigned long long)d2);
        s[0] = s[1] = s[2] = 0;
    }
};

template <typename T>
constexpr size_t tile_dyn_smem() {
    return (size_t)TileCap<T>::REC * sizeof(typename Prec<T>::node4) + TileAcc<T>::bytes(TileCap<T>::ACC);
}

// Geometry of tile T: first row (y0, z0), extent (oy, oz).  Staged rows
// (i, j), 0 <= i <= oy, 0 <= j <= oz, are lattice rows (y0 + i, z0 + j)
// mod (ny, nz), indexed i + (oy + 1) j; the tile's rows (and buckets) are
// those with i < oy, j < oz, indexed i + oy j.
struct TileGeo {
    int ty, tz, y0, z0, oy, oz;
    __host__ __device__ TileGeo(int T, int tiles_y, int ny, int nz) {
        ty = T % tiles_y;
        tz = T / tiles_y;
        y0 = ty * TILE_Y;
        z0 = tz * TILE_Z;
        oy = ny - y0 < TILE_Y ? ny - y0 : TILE_Y;
        oz = nz - z0 < TILE_Z ? nz - z0 : TILE_Z;
    }
    __host__ __device__ int sy() const { return oy + 1; }
    __host__ __device__ int nsr() const { return (oy + 1) * (oz + 1); }
    __host__ __device__ int no() const { return oy * oz; }
};

__device__ __forceinline__ int wrap_row(int y, int n) { return y >= n ? y - n : y; }

// Row kinds: interior rows get transfers from the tile's own particles only;
// a lower-edge row (i = 0 or j = 0) also from the tiles below, through the
// edge accumulator: folded by this tile after waiting (FOLD), or by the
// follow-up kernel when the row lies at y = 0 or z = 0 (WRAP).
enum { ROW_INTERIOR = 0, ROW_FOLD = 1, ROW_WRAP = 2 };
// Tiles below that a tile waits for: bit 0 (ty - 1, tz), bit 1 (ty, tz - 1),
// bit 2 (ty - 1, tz - 1).
enum { DEP_Y = 1, DEP_Z = 2, DEP_YZ = 4 };

// A tile's table: built once per re-ordering (tile_table_kernel), copied in
// one bulk copy by the MD step.  Slots are compact record slots; staged
// record index = slot + rdelta[row], accumulator index = slot + adelta[row]
// (the tile's rows).
struct __align__(16) TileTable {
    int n_rec, n_acc, n_part, staged;  // staged records, the tile's records, particles, fits in shared memory
    int nseg, deps, pad_[2];
    int seg_src[TILE_NSEG], seg_dst[TILE_NSEG], seg_n[TILE_NSEG];  // bulk copies: slot, staged index, count
    int grow[TILE_SR], rdelta[TILE_SR], adelta[TILE_SR];           // staged row: lattice row, index offsets
    int ofirst[TILE_NO], ocnt[TILE_NO], osrc[TILE_NO], aoff[TILE_NO], okind[TILE_NO];  // the tile's rows
    int bstart[TILE_NO], brow[TILE_NO], bij[TILE_NO];  // buckets: first slot, cell row, i | j << 8
    int bpre[TILE_NO + 1];                             // particle entries before bucket b
};
static_assert(sizeof(TileTable) % 16 == 0, "bulk copies move multiples of 16 bytes");

template <typename T>
struct TileArgs {
    typename Prec<T>::real4 *pos_out, *vel_out;  // particle buffer of the new state
    typename Prec<T>::node4 *cact_out;           // record buffer of the new state
    unsigned char *edge;                         // edge accumulator, per compact slot (zero between steps)
    const TileTable *table;                      // per tile
    uint32_t *flag;                              // per tile: MD step (+ 1) whose particles are done
    int32_t *late_rows, *late_count;             // rows whose wait ran out (two lists by MD-step parity)
    int late_cap;
    int tiles_y, n_tiles;
    int32_t *dev_error;  // set if a copy wait gave up
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_expect(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_to_shared(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Wait for phase `parity` of bar, at most TILE_SPIN polls; on a timeout the
// error flag is set and the copies still in flight get a second bounded wait
// before the block goes on (its results are then flagged invalid).
__device__ __forceinline__ void mbar_wait(unsigned long long *bar, uint32_t parity, int32_t *dev_error) {
    int polls = 0;
    while (!mbar_try_wait(bar, parity)) {
        if (++polls > TILE_SPIN) {
            atomicOr(dev_error, 1);
            for (int p2 = 0; p2 < TILE_SPIN && !mbar_try_wait(bar, parity); ++p2) {
            }
            return;
        }
    }
}

// index of the last prefix entry <= v among pre[0..n] (pre non-decreasing,
// pre[0] <= v < pre[n]): the bucket holding entry v
__device__ __forceinline__ int find_run(const int *pre, int n, int v) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= v)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// exclusive warp scan of v over the lanes; returns the total
__device__ __forceinline__ int warp_excl_scan(int lane, int v, int &excl) {
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += u;
    }
    excl = incl - v;
    return __shfl_sync(0xffffffffu, incl, 31);
}

// One warp per tile: the tile's table from the compact-record offsets of
// the rows (arow) and the particle buckets (row_start).
__global__ void __launch_bounds__(256) tile_table_kernel(const int32_t *arow, const int32_t *row_start, int ny,
                                                         int nz, int tiles_y, int n_tiles, int rec_cap, int acc_cap,
                                                         TileTable *table) {
    const int lane = threadIdx.x & 31;
    const int T = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (T >= n_tiles) return;  // whole warps
    const TileGeo G(T, tiles_y, ny, nz);
    const int SY = G.sy(), nsr = G.nsr(), no = G.no();
    TileTable &t = table[T];
    // staged row r = lane
    int first = 0, cnt = 0;
    if (lane < nsr) {
        const int g = wrap_row(G.y0 + lane % SY, ny) + ny * wrap_row(G.z0 + lane / SY, nz);
        first = arow[g];
        cnt = arow[g + 1] - first;
        t.grow[lane] = g;
    }
    int off;
    const int n_rec = warp_excl_scan(lane, cnt, off);
    if (lane < nsr) t.rdelta[lane] = off - first;
    // the tile's row (and bucket) o = lane: (i, j) = (o % oy, o / oy), staged row i + SY j
    const int oi = lane < no ? lane % G.oy : 0, oj = lane < no ? lane / G.oy : 0, r = oi + SY * oj;
    const int ofirst = __shfl_sync(0xffffffffu, first, r), osrc = __shfl_sync(0xffffffffu, off, r);
    const int oc = __shfl_sync(0xffffffffu, cnt, r);
    const int ocnt = lane < no ? oc : 0;
    int aoff;
    const int n_acc = warp_excl_scan(lane, ocnt, aoff);
    int kind = ROW_INTERIOR;
    if (oi == 0 || oj == 0) kind = ((oi == 0 && G.y0 == 0) || (oj == 0 && G.z0 == 0)) ? ROW_WRAP : ROW_FOLD;
    const bool fold = lane < no && kind == ROW_FOLD;
    const unsigned dy = __ballot_sync(0xffffffffu, fold && oi == 0);
    const unsigned dz = __ballot_sync(0xffffffffu, fold && oj == 0);
    const unsigned dyz = __ballot_sync(0xffffffffu, fold && oi == 0 && oj == 0);
    int bcnt = 0;
    if (lane < no) {
        t.ofirst[lane] = ofirst;
        t.ocnt[lane] = ocnt;
        t.osrc[lane] = osrc;
        t.aoff[lane] = aoff;
        t.okind[lane] = kind;
        t.adelta[r] = aoff - ofirst;
        const int gb = (G.y0 + oi) + ny * (G.z0 + oj);
        const int s0 = row_start[gb];
        bcnt = row_start[gb + 1] - s0;
        t.bstart[lane] = s0;
        t.brow[lane] = gb;
        t.bij[lane] = oi | (oj << 8);
    }
    int bpre;
    const int n_part = warp_excl_scan(lane, bcnt, bpre);
    if (lane < no) t.bpre[lane] = bpre;
    if (lane == 0) t.bpre[no] = n_part;
    // contiguous runs of staged rows: one z-line each, split where y wraps to
    // 0; lane 2j + k holds run k of z-line j
    const int nz1 = G.oz + 1;
    int seg_src = 0, seg_dst = 0, seg_n = 0;
    for (int j = 0; j < nz1; ++j) {
        int k = 0, start = 0, n = 0;
        for (int i = 0; i < SY; ++i) {
            const int rr = i + SY * j;
            const int c = __shfl_sync(0xffffffffu, cnt, rr);
            if (i > 0 && G.y0 + i == ny) {  // row 0 is not the slot-order successor of row ny - 1
                const int rs = start + SY * j;
                const int fs = __shfl_sync(0xffffffffu, first, rs), os = __shfl_sync(0xffffffffu, off, rs);
                if (lane == 2 * j) {
                    seg_src = fs;
                    seg_dst = os;
                    seg_n = n;
                }
                k = 1;
                start = i;
                n = 0;
            }
            n += c;
        }
        const int rs = start + SY * j;
        const int fs = __shfl_sync(0xffffffffu, first, rs), os = __shfl_sync(0xffffffffu, off, rs);
        if (lane == 2 * j + k) {
            seg_src = fs;
            seg_dst = os;
            seg_n = n;
        }
    }
    if (lane < TILE_NSEG) {
        t.seg_src[lane] = seg_src;
        t.seg_dst[lane] = seg_dst;
        t.seg_n[lane] = lane < 2 * nz1 ? seg_n : 0;
    }
    if (lane == 0) {
        t.n_rec = n_rec;
        t.n_acc = n_acc;
        t.n_part = n_part;
        t.staged = n_rec <= rec_cap && n_acc <= acc_cap;
        t.nseg = 2 * nz1;
        t.deps = (dy ? DEP_Y : 0) | (dz ? DEP_Z : 0) | (dyz ? DEP_YZ : 0);
    }
}

// One particle of the tile, loaded before the records arrive.
template <typename T>
struct PartRegs {
    typename Prec<T>::real4 R, V;
    int slot, b, id;
};

template <typename T>
__device__ __forceinline__ void load_particle(const PArgs<T> &a, const TileTable &tb, int no, int e, PartRegs<T> &q) {
    q.b = find_run(tb.bpre, no, e);
    q.slot = tb.bstart[q.b] + (e - tb.bpre[q.b]);
    q.R = a.pos4[q.slot];
    q.V = a.vel4[q.slot];
    q.id = a.pid[q.slot];
}

// wait until flag reads `epoch` (at most TILE_SPIN polls 64 ns apart)
__device__ __forceinline__ bool wait_flag(const uint32_t *flag, uint32_t epoch) {
    const volatile uint32_t *f = flag;
    int polls = 0;
    while (*f != epoch) {
        if (++polls > TILE_SPIN) return false;
        __nanosleep(64);
    }
    return true;
}

template <typename T>
__global__ void __launch_bounds__(TILE_THREADS, 3) md_tile_kernel(PArgs<T> a, TileArgs<T> t, int64_t edge_cap) {
    using P = Prec<T>;
    using N4 = typename P::node4;
    using R4 = typename P::real4;
    using fix = typename P::fix;
    using Acc = TileAcc<T>;
    constexpr int REC_CAP = TileCap<T>::REC, ACC_CAP = TileCap<T>::ACC;
    __shared__ TileTable tb;
    __shared__ uint2 words[TILE_SR][TILE_WMAX];
    __shared__ unsigned long long mbar[2];
    __shared__ int s_ok;
    extern __shared__ __align__(128) unsigned char tile_smem[];
    N4 *s_rec = reinterpret_cast<N4 *>(tile_smem);
    unsigned char *s_acc = tile_smem + (size_t)REC_CAP * sizeof(N4);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    const TileGeo G(tile, t.tiles_y, a.ny, a.nz);
    const int oy = G.oy, oz = G.oz, SY = G.sy(), nsr = G.nsr(), no = G.no();

    // (1) the tile's table (bulk copy) and the staged rows' active words
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect(&mbar[0], (uint32_t)sizeof(TileTable));
        bulk_to_shared(&tb, t.table + tile, (uint32_t)sizeof(TileTable), &mbar[0]);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = tid + h * TILE_THREADS, row = k >> 4, w = k & 15;
        if (row < nsr && w < a.occ_words) {
            const int g = wrap_row(G.y0 + row % SY, a.ny) + a.ny * wrap_row(G.z0 + row / SY, a.nz);
            words[row][w] = a.occw[(size_t)g * a.occ_words + w];
        }
    }
    if (tid == 0) mbar_wait(&mbar[0], 0u, t.dev_error);
    __syncthreads();

    // (2) the records (bulk copies), each thread's particle, the sums cleared
    const bool staged = tb.staged != 0;
    const int n_rec = tb.n_rec, n_acc = tb.n_acc, E = tb.n_part;
    if (staged && n_rec > 0 && warp == 0) {
        if (lane == 0) mbar_expect(&mbar[1], (uint32_t)(n_rec * sizeof(N4)));
        __syncwarp();
        if (lane < tb.nseg && tb.seg_n[lane] > 0)
            bulk_to_shared(s_rec + tb.seg_dst[lane], a.cact + tb.seg_src[lane],
                           (uint32_t)(tb.seg_n[lane] * sizeof(N4)), &mbar[1]);
    }
    PartRegs<T> pre;
    if (tid < E) load_particle(a, tb, no, tid, pre);
    if (staged) {
        Acc::clear(s_acc, ACC_CAP, n_acc, tid, TILE_THREADS);
    } else {
        // records from global memory: the tile's old records go to the new
        // buffer first, the transfers are then added there with atomics
        for (int o = warp; o < no; o += TILE_WARPS) {
            const int f = tb.ofirst[o], n = tb.ocnt[o];
            for (int k = lane; k < n; k += 32) t.cact_out[f + k] = a.cact[f + k];
        }
    }
    if (staged && n_rec > 0 && tid == 0) mbar_wait(&mbar[1], 0u, t.dev_error);
    __syncthreads();

    // (3) the MD step of the tile's particles
    const uint32_t md_step = md_step_index(a);
    for (int e = tid; e < E; e += TILE_THREADS) {
        PartRegs<T> q;
        if (e == tid)
            q = pre;
        else
            load_particle(a, tb, no, e, q);
        const int b = q.b, slot = q.slot;
        const int ib = tb.bij[b] & 0xff, jb = tb.bij[b] >> 8;
        const R4 R = q.R;
        R4 V = q.V;
        const uint32_t cell = (uint32_t)P::cell_of(R);
        const uint32_t crow = fdiv(cell, a.fd_nx);
        const bool migrant = crow != (uint32_t)tb.brow[b];
        const int cx = (int)(cell - crow * a.fd_nx.d);
        const int x1 = cx + 1 == a.nx ? 0 : cx + 1;
        bool defer = migrant;
        T ux, uy, uz;
        if (!migrant) {
            interp_u_from(R.x, R.y, R.z, a.fis, ux, uy, uz, [&](int qq, N4 &n0, N4 &n1) {
                const int r = (ib + (qq & 1)) + SY * (jb + (qq >> 1));
                const uint2 w0 = words[r][cx >> 5];
                const uint2 w1 = (x1 >> 5) == (cx >> 5) ? w0 : words[r][x1 >> 5];
                const int s0 = active_slot(w0, cx), s1 = active_slot(w1, x1);
                const int d = tb.rdelta[r];
                const size_t g0 = (size_t)tb.grow[r] * (uint32_t)a.nx;
                if (s0 >= 0)
                    n0 = staged ? s_rec[s0 + d] : a.cact[s0];
                else
                    n0 = a.node[g0 + cx];
                if (s1 >= 0)
                    n1 = staged ? s_rec[s1 + d] : a.cact[s1];
                else
                    n1 = a.node[g0 + x1];
                defer = defer || s0 < 0 || s1 < 0;
            });
        } else {
            interp_u(a, cell_xyz(cell, a.fd_nx, a.fd_ny), R.x, R.y, R.z, ux, uy, uz);
        }
        T Fx, Fy, Fz;
        coupling_force_id(a, (uint32_t)q.id, md_step, V, ux, uy, uz, Fx, Fy, Fz);
        {
            // velocity Verlet with F held fixed over the step (no
            // conservative forces on this path)
            const T hm = a.half_dt * V.w;  // V.w = 1 / mass
            V.x = fma(hm, Fx, V.x);
            V.y = fma(hm, Fy, V.y);
            V.z = fma(hm, Fz, V.z);
            const int cz = (int)fdiv(crow, a.fd_ny);
            int cy = (int)crow - cz * a.ny, cxn = cx, czn = cz;
            T fx = R.x, fy = R.y, fz = R.z;
            advance(fx, cxn, a.dt, V.x, a.nx);
            advance(fy, cy, a.dt, V.y, a.ny);
            advance(fz, czn, a.dt, V.z, a.nz);
            V.x = fma(hm, Fx, V.x);
            V.y = fma(hm, Fy, V.y);
            V.z = fma(hm, Fz, V.z);
            t.pos_out[slot] = P::make_pos(fx, fy, fz, cxn + (int64_t)a.nx * (cy + (int64_t)a.ny * czn));
            t.vel_out[slot] = V;
        }
        if (defer) {
            a.old4[slot] = R;
            a.fc4[slot] = P::make4(Fx, Fy, Fz, T(0));
            a.migrant_slot[(int64_t)a.mig_par * a.np_cap + atomicAdd(a.migrant_count + a.mig_par, 1)] = slot;
            continue;
        }
        // the transfers -delta_k dt F: the tile's rows in shared memory, the
        // rows above the tile into the edge accumulator
        const T sx = Fx * a.neg_scale_dt, sy = Fy * a.neg_scale_dt, sz = Fz * a.neg_scale_dt;
        const T wx[2] = {T(1) - R.x, R.x};
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            const int ii = ib + (qq & 1), jj = jb + (qq >> 1);
            const int r = ii + SY * jj;
            const bool own = ii < oy && jj < oz;
            const T wy = (qq & 1) ? R.y : T(1) - R.y;
            const T wz = (qq >> 1) ? R.z : T(1) - R.z;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int xn = h ? x1 : cx;
                const T dk = wx[h] * wy * wz;  // the corner weight delta_k of Eq. (5)
                const fix vx = P::to_fix_neg(dk, sx), vy = P::to_fix_neg(dk, sy), vz = P::to_fix_neg(dk, sz);
                const int sl = active_slot(words[r][xn >> 5], xn);
                if (!own)
                    Acc::add(t.edge, (int)edge_cap, sl, vx, vy, vz);
                else if (staged)
                    Acc::add(s_acc, ACC_CAP, sl + tb.adelta[r], vx, vy, vz);
                else
                    P::add_transfer(&t.cact_out[sl], vx, vy, vz);
            }
        }
    }
    // (4) publish: the tile's transfers to the rows above are in
    __syncthreads();
    const uint32_t epoch = md_step + 1u;
    if (tid == 0) {
        __threadfence();
        atomicExch(&t.flag[tile], epoch);
        // the tiles below whose transfers reach this tile's lower-edge rows
        bool ok = true;
        if (tb.deps & DEP_Y) ok = ok && wait_flag(t.flag + tile - 1, epoch);
        if (tb.deps & DEP_Z) ok = ok && wait_flag(t.flag + tile - t.tiles_y, epoch);
        if (tb.deps & DEP_YZ) ok = ok && wait_flag(t.flag + tile - t.tiles_y - 1, epoch);
        __threadfence();
        s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    const bool ok = s_ok != 0;
    // (5) the tile's records, old value plus the sums (and, for the
    // lower-edge rows, the edge accumulator), into the new buffer; one warp
    // per row
    for (int o = warp; o < no; o += TILE_WARPS) {
        const int f = tb.ofirst[o], n = tb.ocnt[o], kind = tb.okind[o];
        const bool fold = kind == ROW_FOLD && ok;
        if (kind == ROW_FOLD && !ok && lane == 0) {
            // left to the follow-up kernel
            const int g = (G.y0 + (tb.bij[o] & 0xff)) + a.ny * (G.z0 + (tb.bij[o] >> 8));
            const int k = atomicAdd(t.late_count + a.mig_par, 1);
            if (k < t.late_cap) t.late_rows[(int64_t)a.mig_par * t.late_cap + k] = g;
            else atomicOr(t.dev_error, 2);
        }
        if (staged) {
            const int src = tb.osrc[o], a0 = tb.aoff[o];
            for (int k = lane; k < n; k += 32) {
                N4 rec = s_rec[src + k];
                Acc::take(s_acc, ACC_CAP, a0 + k, rec);
                if (fold) Acc::take_clear_global(t.edge, edge_cap, f + k, rec);
                t.cact_out[f + k] = rec;
            }
        } else if (fold) {
            for (int k = lane; k < n; k += 32) {
                N4 rec = t.cact_out[f + k];
                Acc::take_clear_global(t.edge, edge_cap, f + k, rec);
                t.cact_out[f + k] = rec;
            }
        }
    }
}

// After the tiles: the edge accumulator of the rows at y = 0 or z = 0 (their
// lower neighbours wrap to the far end of the grid) and of the rows whose
// wait ran out, folded into the new records with atomics; then the listed
// particles spread with atomics (as migrant_spread_kernel).
template <typename T>
__global__ void __launch_bounds__(256) md_tile_finish_kernel(PArgs<T> a, TileArgs<T> t, const int32_t *arow,
                                                             int64_t edge_cap) {
    using Acc = TileAcc<T>;
    const int par = a.mig_par;
    const int n_fix = a.nz + a.ny - 1;
    const int n_late = min(t.late_count[par], t.late_cap);
    const int warps = (int)(gridDim.x * blockDim.x) >> 5;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    for (int k = gw; k < n_fix + n_late; k += warps) {
        const int g = k < a.nz ? a.ny * k
                               : (k < n_fix ? k - a.nz + 1 : t.late_rows[(int64_t)par * t.late_cap + (k - n_fix)]);
        const int f = arow[g], n = arow[g + 1] - f;
        for (int s = lane; s < n; s += 32) Acc::fold_atomic(t.edge, edge_cap, f + s, &t.cact_out[f + s]);
    }
    // the lists of the next step start empty
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.migrant_count[par ^ 1] = 0;
        t.late_count[par ^ 1] = 0;
    }
    const int n = a.migrant_count[par];
    const int32_t *list = a.migrant_slot + (int64_t)par * a.np_cap;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        spread_particle_atomic(a, (int64_t)list[i]);
}

template <typename T>
cudaError_t md_tile_setup() {
    return cudaFuncSetAttribute(md_tile_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_dyn_smem<T>());
}

}  // namespace lbmd

// Whether the lattice suits the tiled step (variant B): rows of at most 512
// nodes, at least TILE + 2 rows in y and z (the staged rows of a tile and the
// rows the follow-up folds are all distinct).
bool md_tile_geometry(const lbmd_ctx *ctx) {
    return ctx->p.variant == LBMD_VARIANT_B && ctx->p.nx <= 32 * lbmd::TILE_WMAX && ctx->p.ny >= lbmd::TILE_Y + 2 &&
           ctx->p.nz >= lbmd::TILE_Z + 2;
}

// Whether the tiled step can run this context's MD steps: the geometry, the
// START integrator, ideal particles, and the tiles' buffers allocated.
bool md_tile_supported(const lbmd_ctx *ctx) {
    return md_tile_geometry(ctx) && ctx->tile_table[0] && ctx->p.integrator == LBMD_INTEGRATOR_START &&
           !has_cons(ctx);
}

// Expected records of a tile's staged rows for uniformly spread particles
// (a node is active with probability 1 - exp(-8 n_p / N)), against the
// shared-memory capacity: AUTO takes the tiled step only when it fits.
bool md_tile_expected_to_fit(const lbmd_ctx *ctx) {
    const double f = 1.0 - std::exp(-8.0 * (double)ctx->np / (double)ctx->N);
    const double staged = (double)lbmd::TILE_SR * ctx->p.nx * f;
    const int cap = ctx->p.precision == LBMD_FP64 ? lbmd::TileCap<double>::REC : lbmd::TileCap<float>::REC;
    return staged <= 0.9 * cap;
}

int md_tile_count(const lbmd_ctx *ctx) {
    return ((ctx->p.ny + lbmd::TILE_Y - 1) / lbmd::TILE_Y) * ((ctx->p.nz + lbmd::TILE_Z - 1) / lbmd::TILE_Z);
}

size_t md_tile_table_bytes(const lbmd_ctx *ctx) { return (size_t)md_tile_count(ctx) * sizeof(lbmd::TileTable); }

// bytes of the edge accumulator per compact record slot
size_t md_tile_edge_bytes(const lbmd_ctx *ctx) {
    return ctx->p.precision == LBMD_FP64 ? lbmd::TileAcc<double>::bytes(1) : lbmd::TileAcc<float>::bytes(1);
}

// rows whose edge accumulator a tile may leave to the follow-up kernel
int md_tile_late_cap(const lbmd_ctx *ctx) { return md_tile_count(ctx) * (lbmd::TILE_Y + lbmd::TILE_Z - 1); }

cudaError_t md_tile_setup_kernels(lbmd_ctx *ctx) {
    return ctx->p.precision == LBMD_FP64 ? lbmd::md_tile_setup<double>() : lbmd::md_tile_setup<float>();
}

// The tiles' tables of active set `set` from its row offsets and the current
// particle buckets (after every re-ordering).
cudaError_t md_tile_build_table(lbmd_ctx *ctx, int set) {
    if (!ctx->tile_table[set]) return cudaSuccess;
    const int tiles_y = (ctx->p.ny + lbmd::TILE_Y - 1) / lbmd::TILE_Y;
    const int n_tiles = md_tile_count(ctx);
    const bool f64 = ctx->p.precision == LBMD_FP64;
    lbmd::tile_table_kernel<<<(n_tiles + 7) / 8, 256, 0, ctx->stream>>>(
        ctx->arow[set], ctx->row_start, ctx->p.ny, ctx->p.nz, tiles_y, n_tiles,
        f64 ? lbmd::TileCap<double>::REC : lbmd::TileCap<float>::REC,
        f64 ? lbmd::TileCap<double>::ACC : lbmd::TileCap<float>::ACC,
        static_cast<lbmd::TileTable *>(ctx->tile_table[set]));
    return cudaGetLastError();
}

// One tiled MD step: the tiles, then the follow-up (edge rows at the wrap,
// timed-out rows, listed particles).  Positions, velocities and records go to
// the other buffers; the caller flips them.
template <typename T>
cudaError_t md_tile_step(lbmd_ctx *ctx, const lbmd::PArgs<T> &a) {
    using P = lbmd::Prec<T>;
    lbmd::TileArgs<T> t;
    const int o = ctx->pv ^ 1;
    t.pos_out = static_cast<typename P::real4 *>(ctx->pos4[o]);
    t.vel_out = static_cast<typename P::real4 *>(ctx->vel4[o]);
    t.cact_out = static_cast<typename P::node4 *>(active_records_other(ctx));
    t.edge = static_cast<unsigned char *>(ctx->edge_acc);
    t.table = static_cast<const lbmd::TileTable *>(ctx->tile_table[ctx->lb_step & 1]);
    t.flag = ctx->tile_flag;
    t.late_rows = ctx->late_rows;
    t.late_count = ctx->late_count;
    t.late_cap = md_tile_late_cap(ctx);
    t.tiles_y = (ctx->p.ny + lbmd::TILE_Y - 1) / lbmd::TILE_Y;
    t.n_tiles = md_tile_count(ctx);
    t.dev_error = ctx->dev_error;
    lbmd::md_tile_kernel<T>
        <<<t.n_tiles, lbmd::TILE_THREADS, lbmd::tile_dyn_smem<T>(), ctx->stream>>>(a, t, ctx->cact_cap);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lbmd::PArgs<T> m = a;
    m.cact = m.cact_acc = t.cact_out;  // the listed particles spread into the new records
    lbmd::md_tile_finish_kernel<T><<<ctx->sm_count, 256, 0, ctx->stream>>>(m, t, ctx->arow[ctx->lb_step & 1],
                                                                         ctx->cact_cap);
    return cudaGetLastError();
}

template cudaError_t md_tile_step<float>(lbmd_ctx *, const lbmd::PArgs<float> &);
template cudaError_t md_tile_step<double>(lbmd_ctx *, const lbmd::PArgs<double> &);
