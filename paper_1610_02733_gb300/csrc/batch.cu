// batch.cu -- batched replicas: many independent periodic boxes advanced
// together on one GPU.  Each replica is a complete problem of its own (its
// lattice, particles, friction zeta, MD steps per LB step m, variant and
// Philox key) and evolves exactly as a single-box context with the same
// parameters would: the kernels below run the same collision (lb_core.cuh),
// the same interpolation, noise, integrator and fixed-point transfers
// (particle_core.cuh) with per-replica offsets.  The paper's temperature
// experiment (Sec. 4: particle temperature against zeta, m and dt, variants A
// and B) needs many such boxes; one launch per phase covers all of them.
//
// Schedule.  All replicas make one MD step per tick; replica r makes its LB
// step after every m_r-th tick.  A period of P = lcm(m_r) ticks repeats, and
// is captured once into a CUDA graph: per tick the couple kernel (every
// particle), the transfer kernel (variant-B particles), and, for the replicas
// whose LB step is due, the collide and moments kernels driven by a
// precomputed table of work items (replica, first node); the moments kernel
// also advances the LB step counters.
//
// Transfers are integer atomics on the replica's node field (B) or transfer
// accumulator (A): the boxes are small enough to stay in L2, and integer sums
// keep the result independent of the order (bitwise reproducible).
//
// Stability.  Explicit friction is unstable for zeta dt / m >~ 2 (the
// velocity map v -> v (1 - zeta dt / m) overshoots); such replicas are not
// clamped: a replica whose particle speed leaves any physical range (|v| > 1
// lattice unit per time unit, or not finite) is flagged unstable and frozen,
// and reported as such.
//
// Autotuner.  The block sizes of the node kernels (nodes per item) and of
// the particle kernels are chosen by timing each candidate with CUDA events
// on this batch (node kernels at creation on the rest state, which is then
// restored; particle kernels at the first run, on copies of the state).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "lb_core.cuh"
#include "lbmd_ctx.h"
#include "lbmd_device.cuh"
#include "particle_core.cuh"
#include "convert.cuh"

namespace lbmd {

constexpr int BATCH_MAX_EDGE = 512;
constexpr int64_t BATCH_MAX_PERIOD = 256;
constexpr int BATCH_VMAX2 = 1;  // |v|^2 beyond which a replica counts as unstable
constexpr int BATCH_LB_MAX_NODES = 256;  // nodes per work item of the LB kernels, at most
constexpr int BATCH_LB_MAX_THREADS = BATCH_LB_MAX_NODES + 32;

// Per-replica constants, one entry per replica in device memory.
template <typename T>
struct BRep {
    int nx, ny, nz, n_sub;
    int variant, np;
    int64_t node_off;  // first node of the replica in the node arrays (populations: 19 x that)
    int64_t part_off;  // first particle slot of the replica
    FastDiv fd_nx, fd_ny;
    uint32_t key0, key1;
    T zeta, dt, half_dt, amp, neg_scale_dt;
};

template <typename T>
struct BArgs {
    using P = Prec<T>;
    const BRep<T> *rep;
    const int32_t *prep;  // replica of every particle slot
    int64_t n_slots;
    typename P::real4 *pos4, *vel4, *fc4, *old4;
    typename P::node4 *node, *jacc;
    const unsigned long long *lb_step;
    int *unstable;
    int tick;  // MD step within the period
    T fis;     // 1 / fixed-point scale of the momentum density (shared rho0)
};

template <typename T>
struct BLbArgs {
    const BRep<T> *rep;
    const int2 *work;  // per item: replica, first node
    int64_t n_items;
    T *f0, *f1;        // population buffers: replica r's 19 N_r values at 19 node_off
    typename Prec<T>::node4 *node, *jacc;
    unsigned long long *lb_step;
    const int *unstable;
    unsigned *items_done;  // per replica: items of the moments kernel taken so far
    int advance;           // the moments kernel advances the LB step counters
    int nodes_per_block;
    T fs, fis;             // fixed-point scale of the momentum density and its inverse
    // members read by collide()
    T gamma_bulk, gamma_shear, gamma_ghost;
    T amp16[Q];
    int noisy;
};

// Node records read through L2 only (ld.global.cg), for data that other
// blocks of the same launch write.
__device__ __forceinline__ int4 load_cg(const int4 *p) { return __ldcg(p); }
__device__ __forceinline__ L4 load_cg(const L4 *p) {
    const longlong2 a = __ldcg(reinterpret_cast<const longlong2 *>(p));
    const longlong2 b = __ldcg(reinterpret_cast<const longlong2 *>(p) + 1);
    L4 n;
    n.x = a.x;
    n.y = a.y;
    n.z = b.x;
    n.w = b.y;
    return n;
}

// One MD step of the particle in slot p (replica r, index `local` within
// it): interpolation (Eq. (5)), friction and random force (Eq. (4)) with the
// Philox counter of the replica's MD step lb_step m_r + cyc (cyc: the MD step
// within the replica's LB cycle), velocity Verlet with the force held over
// the step; variant A hands the transfer straight to the accumulator,
// variant B keeps the start position and the force for the transfer.  Shared
// by both schedules of lbmd_batch_run, so that they do the same arithmetic.
template <typename T, bool CG = false>
__device__ __forceinline__ void batch_couple_particle(const BArgs<T> &a, int64_t p, int r, const BRep<T> &rp,
                                                      int64_t local, unsigned long long lb_step, int cyc) {
    using P = Prec<T>;
    const typename P::real4 R = a.pos4[p];
    typename P::real4 V = a.vel4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), rp.fd_nx, rp.fd_ny);
    uint32_t idx[8];
    T delta[8];
    corners(c, R.x, R.y, R.z, rp.nx, rp.ny, rp.nz, idx, delta);
    const typename P::node4 *node = a.node + rp.node_off;
    T ux = T(0), uy = T(0), uz = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const typename P::node4 n = CG ? load_cg(node + idx[k]) : node[idx[k]];
        const T w = delta[k] / P::rho_of(n);
        ux = fma(w, P::from_fix(P::jx_of(n), a.fis), ux);
        uy = fma(w, P::from_fix(P::jy_of(n), a.fis), uy);
        uz = fma(w, P::from_fix(P::jz_of(n), a.fis), uz);
    }
    T Fx = -rp.zeta * (V.x - ux), Fy = -rp.zeta * (V.y - uy), Fz = -rp.zeta * (V.z - uz);
    if (rp.amp != T(0)) {
        const uint32_t md_step = (uint32_t)(lb_step * (unsigned long long)rp.n_sub + (unsigned)cyc);
        const U4 rnd = philox4x32_10(U4{(uint32_t)local, md_step, 1u, 0u}, rp.key0, rp.key1);
        Fx = fma(rp.amp, unit_uniform<T>(rnd.x), Fx);
        Fy = fma(rp.amp, unit_uniform<T>(rnd.y), Fy);
        Fz = fma(rp.amp, unit_uniform<T>(rnd.z), Fz);
    }
    const T hm = rp.half_dt * V.w;
    V.x = fma(hm, Fx, V.x);
    V.y = fma(hm, Fy, V.y);
    V.z = fma(hm, Fz, V.z);
    T fx = R.x, fy = R.y, fz = R.z;
    int cx = c.x, cy = c.y, cz = c.z;
    advance(fx, cx, rp.dt, V.x, rp.nx);
    advance(fy, cy, rp.dt, V.y, rp.ny);
    advance(fz, cz, rp.dt, V.z, rp.nz);
    V.x = fma(hm, Fx, V.x);
    V.y = fma(hm, Fy, V.y);
    V.z = fma(hm, Fz, V.z);
    if (!(V.x * V.x + V.y * V.y + V.z * V.z <= T(BATCH_VMAX2))) {
        a.unstable[r] = 1;  // explicit friction diverged: freeze the replica
        return;
    }
    a.pos4[p] = P::make_pos(fx, fy, fz, cx + (int64_t)rp.nx * (cy + (int64_t)rp.ny * cz));
    a.vel4[p] = V;
    if (rp.variant == LBMD_VARIANT_A) {
        spread_to<T>(a.jacc + rp.node_off, idx, delta, Fx * rp.neg_scale_dt, Fy * rp.neg_scale_dt,
                     Fz * rp.neg_scale_dt);
    } else {
        a.old4[p] = R;
        a.fc4[p] = P::make4(Fx, Fy, Fz, T(0));
    }
}

// Variant B: the transfers of the particle in slot p (Eqs. (7), (8)), once
// every particle of its replica has read the node field.
template <typename T>
__device__ __forceinline__ void batch_transfer_particle(const BArgs<T> &a, int64_t p, const BRep<T> &rp) {
    using P = Prec<T>;
    const typename P::real4 R = a.old4[p];
    const typename P::real4 F = a.fc4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), rp.fd_nx, rp.fd_ny);
    uint32_t idx[8];
    T delta[8];
    corners(c, R.x, R.y, R.z, rp.nx, rp.ny, rp.nz, idx, delta);
    spread_to<T>(a.node + rp.node_off, idx, delta, F.x * rp.neg_scale_dt, F.y * rp.neg_scale_dt,
                 F.z * rp.neg_scale_dt);
}

// One MD step of every particle (per-tick schedule).
template <typename T>
__global__ void __launch_bounds__(256) batch_couple_kernel(BArgs<T> a) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_slots) return;
    // the slot's replica (every slot is allocated; an unused one is simply
    // not used)
    const int r = a.prep[p];
    const BRep<T> &rp = a.rep[r];
    const int64_t local = p - rp.part_off;
    if (local >= rp.np || a.unstable[r]) return;
    batch_couple_particle(a, p, r, rp, local, a.lb_step[r], a.tick % rp.n_sub);
}

// Variant B: the transfers of the MD step (per-tick schedule), once every
// particle has read the node field.
template <typename T>
__global__ void __launch_bounds__(256) batch_transfer_kernel(BArgs<T> a) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_slots) return;
    const int r = a.prep[p];
    const BRep<T> &rp = a.rep[r];
    if (rp.variant != LBMD_VARIANT_B || p - rp.part_off >= rp.np || a.unstable[r]) return;
    batch_transfer_particle(a, p, rp);
}

// The LB kernels walk their work table with persistent blocks: block b takes
// items b, b + G, b + 2G, ... (G = grid size).  Every block has one warp more
// than it has nodes per item; that warp fetches the headers of the coming
// items (work entry, the replica's constants and LB step counter) into shared
// memory while the others process the current item, so no block waits on
// that chain of dependent loads.  It reads the work entries of 32 of the
// block's items at a time, with their replicas' frozen flags, and skips the
// items of frozen replicas.
template <typename T>
struct BItem {
    BRep<T> rep;
    unsigned long long step;  // the replica's LB step counter
    int r, first;             // replica (< 0: the block has no further item), first node
};
static_assert(sizeof(BRep<float>) % 4 == 0 && sizeof(BRep<double>) % 4 == 0, "BRep is copied by words");

// State of the prefetch warp: the next window of 32 items, and in the current
// one each lane's work entry and the mask of the live items not yet taken.
struct ItemWindow {
    int64_t next;
    int2 w;
    unsigned live;
};

// The prefetch warp: the next live item of this block into *out (r < 0 once
// the table is exhausted).
template <typename T>
__device__ __forceinline__ void fetch_item(const BLbArgs<T> &a, ItemWindow &win, BItem<T> *out) {
    const int lane = (int)(threadIdx.x & 31u);
    const int64_t stride = gridDim.x;
    while (win.live == 0u) {
        if (win.next >= a.n_items) {
            if (lane == 0) out->r = -1;
            return;
        }
        const int64_t it = win.next + lane * stride;
        win.w = make_int2(-1, 0);
        int live = 0;
        if (it < a.n_items) {
            win.w = a.work[it];
            live = !a.unstable[win.w.x];
        }
        win.live = __ballot_sync(0xffffffffu, live);
        win.next += 32 * stride;
    }
    const int src = __ffs(win.live) - 1;
    win.live &= win.live - 1u;
    const int r = __shfl_sync(0xffffffffu, win.w.x, src);
    const int first = __shfl_sync(0xffffffffu, win.w.y, src);
    const uint32_t *rw = reinterpret_cast<const uint32_t *>(a.rep + r);
    uint32_t *ow = reinterpret_cast<uint32_t *>(&out->rep);
    for (int k = lane; k < (int)(sizeof(BRep<T>) / 4); k += 32) ow[k] = rw[k];
    if (lane == 0) {
        out->step = a.lb_step[r];
        out->r = r;
        out->first = first;
    }
}

// Asynchronous copies global -> shared memory (cp.async, BYTES = 4, 8 or
// 16, both addresses aligned to BYTES): a thread stages the values of its
// node of the next item while it computes the current one, and waits only
// for its own copies.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most the newest committed group is still in flight
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Shared memory of an LB block: two buffers of the staged populations of an
// item (population i of node slot t at [buf][i][t]) and, for the collide, of
// its node records.
template <typename T>
size_t lb_smem_bytes(int nodes_per_block, bool with_node) {
    return (size_t)2 * nodes_per_block * (Q * sizeof(T) + (with_node ? sizeof(typename Prec<T>::node4) : 0));
}

// The item loop shared by the LB kernels.  Per item k of this block: the
// prefetch warp fetches the header of item k + 2; every other thread issues
// the copies of its node of item k + 1 (issue(item, node, buf)), waits for
// its copies of item k and runs body(item, node, buf) on them, then thread 0
// runs once(item).  Three header slots and two staging buffers rotate.
template <typename T, typename Issue, typename Body, typename Once>
__device__ __forceinline__ void for_items(const BLbArgs<T> &a, Issue issue, Body body, Once once) {
    __shared__ BItem<T> s_item[3];
    const bool pre = threadIdx.x >= (unsigned)a.nodes_per_block;
    ItemWindow win{(int64_t)blockIdx.x, make_int2(-1, 0), 0u};
    if (pre) fetch_item(a, win, &s_item[0]);
    __syncthreads();
    if (s_item[0].r < 0) return;
    if (pre) {
        fetch_item(a, win, &s_item[1]);
    } else {
        issue(s_item[0], (int64_t)s_item[0].first + threadIdx.x, 0);
        cp_async_commit();
    }
    __syncthreads();
    int slot = 0;
    for (int k = 0;; ++k) {
        const BItem<T> &cur = s_item[slot];
        if (cur.r < 0) break;
        const int s1 = slot == 2 ? 0 : slot + 1, s2 = s1 == 2 ? 0 : s1 + 1;
        const BItem<T> &nxt = s_item[s1];
        if (pre) {
            fetch_item(a, win, &s_item[s2]);
        } else {
            if (nxt.r >= 0) issue(nxt, (int64_t)nxt.first + threadIdx.x, (k + 1) & 1);
            cp_async_commit();
            cp_async_wait_prev();
            body(cur, (int64_t)cur.first + threadIdx.x, k & 1);
            if (threadIdx.x == 0) once(cur);
        }
        __syncthreads();
        slot = s1;
    }
    if (!pre) cp_async_wait_all();
}

// A staged node record, read from shared memory in 16-byte pieces.
template <typename T>
__device__ __forceinline__ typename Prec<T>::node4 staged_node(const unsigned char *p) {
    typename Prec<T>::node4 n;
    const int4 *src = reinterpret_cast<const int4 *>(p);
    int4 *dst = reinterpret_cast<int4 *>(&n);
#pragma unroll
    for (int h = 0; h < (int)(sizeof(n) / 16); ++h) dst[h] = src[h];
    return n;
}

// Collide node `loc` of replica rp at its LB step `step` (Eq. (3): moments,
// the transfer of the cycle from the node record (B) or the accumulator
// (A), MRT collision with noise) from its populations f and record n, and
// push the result to the neighbours in the other buffer.  Shared by both
// schedules of lbmd_batch_run.
template <typename T, bool RELAX_FULL>
__device__ __forceinline__ void batch_collide_node(const BLbArgs<T> &a, const BRep<T> &rp, unsigned long long step,
                                                   int64_t loc, T (&f)[Q], const typename Prec<T>::node4 &n) {
    using P = Prec<T>;
    using N4 = typename P::node4;
    const int64_t N = (int64_t)rp.nx * rp.ny * rp.nz;
    T *__restrict__ fout = ((step & 1ull) ? a.f0 : a.f1) + 19 * rp.node_off;
    const uint32_t u = (uint32_t)loc;
    const uint32_t row = fdiv(u, rp.fd_nx);
    const int x = (int)(u - row * rp.fd_nx.d);
    const int z = (int)fdiv(row, rp.fd_ny);
    const int y = (int)(row - (uint32_t)z * rp.fd_ny.d);
    T rho, jx, jy, jz;
    node_moments(f, rho, jx, jy, jz);
    T Fx, Fy, Fz;
    if (rp.variant == LBMD_VARIANT_B) {
        Fx = P::from_fix(P::jx_of(n) - P::to_fix(jx, a.fs), a.fis);
        Fy = P::from_fix(P::jy_of(n) - P::to_fix(jy, a.fs), a.fis);
        Fz = P::from_fix(P::jz_of(n) - P::to_fix(jz, a.fs), a.fis);
    } else {
        Fx = P::from_fix(P::jx_of(n), a.fis);
        Fy = P::from_fix(P::jy_of(n), a.fis);
        Fz = P::from_fix(P::jz_of(n), a.fis);
        N4 zero;
        zero.x = zero.y = zero.z = zero.w = 0;
        a.jacc[rp.node_off + loc] = zero;
    }
    collide<T, RELAX_FULL>(f, rho, rho, jx, jy, jz, Fx, Fy, Fz, a, rp.key0, rp.key1, u, (uint32_t)step);
    const int nx = rp.nx, ny = rp.ny, nz = rp.nz;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const int X[3] = {xm, x, xp}, Y[3] = {ym, y, yp}, Z[3] = {zm, z, zp};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int64_t d = (int64_t)X[CX(i) + 1] + (int64_t)nx * (Y[CY(i) + 1] + (int64_t)ny * Z[CZ(i) + 1]);
        fout[(int64_t)i * N + d] = f[i];
    }
}

// Post-stream moments (Eqs. (1), (2)) of node `loc` of replica rp from its
// populations fl -> node field.  Shared by both schedules.
template <typename T>
__device__ __forceinline__ void batch_moments_node(const BLbArgs<T> &a, const BRep<T> &rp, int64_t loc,
                                                   const T (&fl)[Q]) {
    using P = Prec<T>;
    T rho, jx, jy, jz;
    node_moments(fl, rho, jx, jy, jz);
    a.node[rp.node_off + loc] = P::pack(rho, P::to_fix(jx, a.fs), P::to_fix(jy, a.fs), P::to_fix(jz, a.fs));
}

// LB collide and push of the due replicas (Eq. (3)) on the nodes
// [first, first + nodes_per_block) of each item.  Staged per node: the 19
// populations and the node record (variant B) or the transfer accumulator
// (variant A).
template <typename T, bool RELAX_FULL>
__global__ void __launch_bounds__(BATCH_LB_MAX_THREADS, sizeof(T) == 4 ? 4 : 2) batch_collide_kernel(BLbArgs<T> a) {
    using P = Prec<T>;
    using N4 = typename P::node4;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nb = a.nodes_per_block, t = (int)threadIdx.x;
    unsigned char *s_node = smem;                                         // [2][nb] records
    T *s_pop = reinterpret_cast<T *>(smem + (size_t)2 * nb * sizeof(N4));  // [2][Q][nb]
    auto issue = [&](const BItem<T> &it, int64_t loc, int buf) {
        const BRep<T> &rp = it.rep;
        const int64_t N = (int64_t)rp.nx * rp.ny * rp.nz;
        if (loc >= N) return;
        const T *fin = ((it.step & 1ull) ? a.f1 : a.f0) + 19 * rp.node_off + loc;
        T *dst = s_pop + (size_t)buf * Q * nb + t;
#pragma unroll
        for (int i = 0; i < Q; ++i) cp_async<sizeof(T)>(dst + i * nb, fin + i * N);
        const N4 *rec = (rp.variant == LBMD_VARIANT_B ? a.node : a.jacc) + rp.node_off + loc;
        unsigned char *dn = s_node + ((size_t)buf * nb + t) * sizeof(N4);
#pragma unroll
        for (int h = 0; h < (int)(sizeof(N4) / 16); ++h)
            cp_async<16>(dn + 16 * h, reinterpret_cast<const unsigned char *>(rec) + 16 * h);
    };
    auto body = [&](const BItem<T> &it, int64_t loc, int buf) {
        const BRep<T> &rp = it.rep;
        const int64_t N = (int64_t)rp.nx * rp.ny * rp.nz;
        if (loc >= N) return;
        const T *src = s_pop + (size_t)buf * Q * nb + t;
        T f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = src[i * nb];
        const N4 n = staged_node<T>(s_node + ((size_t)buf * nb + t) * sizeof(N4));
        batch_collide_node<T, RELAX_FULL>(a, rp, it.step, loc, f, n);
    };
    for_items(a, issue, body, [](const BItem<T> &) {});
}

// Post-stream moments of the due replicas -> node field.  With advance set,
// the block that takes the last item of a replica advances the replica's LB
// step counter: every item of the replica has been fetched, and so has read
// the counter, by then.
template <typename T>
__global__ void __launch_bounds__(BATCH_LB_MAX_THREADS) batch_moments_kernel(BLbArgs<T> a) {
    using P = Prec<T>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nb = a.nodes_per_block, t = (int)threadIdx.x;
    T *s_pop = reinterpret_cast<T *>(smem);  // [2][Q][nb]
    auto issue = [&](const BItem<T> &it, int64_t loc, int buf) {
        const BRep<T> &rp = it.rep;
        const int64_t N = (int64_t)rp.nx * rp.ny * rp.nz;
        if (loc >= N) return;
        const T *f = (((it.step + 1ull) & 1ull) ? a.f1 : a.f0) + 19 * rp.node_off + loc;
        T *dst = s_pop + (size_t)buf * Q * nb + t;
#pragma unroll
        for (int i = 0; i < Q; ++i) cp_async<sizeof(T)>(dst + i * nb, f + i * N);
    };
    auto body = [&](const BItem<T> &it, int64_t loc, int buf) {
        const BRep<T> &rp = it.rep;
        const int64_t N = (int64_t)rp.nx * rp.ny * rp.nz;
        if (loc >= N) return;
        const T *src = s_pop + (size_t)buf * Q * nb + t;
        T fl[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) fl[i] = src[i * nb];
        batch_moments_node(a, rp, loc, fl);
    };
    auto advance = [&](const BItem<T> &it) {
        if (!a.advance) return;
        const int64_t N = (int64_t)it.rep.nx * it.rep.ny * it.rep.nz;
        const unsigned items = (unsigned)((N + a.nodes_per_block - 1) / a.nodes_per_block);
        if (atomicAdd(&a.items_done[it.r], 1u) == items - 1u) {
            a.items_done[it.r] = 0u;
            a.lb_step[it.r] = it.step + 1ull;
        }
    };
    for_items(a, issue, body, advance);
}

// Persistent schedule (LBMD_BATCH_PERSISTENT).  One launch runs the `ticks`
// MD steps of a lbmd_batch_run call for every replica.  The grid is a set of
// thread-block clusters (as many as fit on the GPU at once); a cluster takes
// replicas one at a time from a queue (heaviest first) and runs all the
// ticks of the replica it holds, separating the phases of a tick with cluster
// barriers (hardware barriers of blocks that the GPU schedules together, so
// no wait can hang): the particles' MD step, [barrier], the variant-B
// transfers, [barrier], and when the replica's LB step is due the collide and
// push, [barrier], the post-stream moments, [barrier].  Replicas are
// independent, so nothing synchronises the whole grid: a cluster that holds a
// small replica simply takes the next one.  Every node and particle goes
// through the same per-node and per-particle functions as in the per-tick
// schedule.
template <typename T>
struct BPersist {
    BArgs<T> p;             // particle arrays (p.tick unused)
    BLbArgs<T> l;           // LB arrays and collision constants (work table unused)
    const int32_t *order;   // replicas, heaviest first
    int R;
    int ticks;              // MD steps of this launch
    int cluster;            // blocks per cluster
    long long *tick0;       // first MD step of the launch; the last cluster to finish advances it
    unsigned *queue;        // [0]: next index into order, [1]: clusters done (both zeroed before the launch)
    int32_t *taken;         // per cluster, two slots by iteration parity: the index it took
};

// barrier of all threads of the cluster; release / acquire at cluster scope
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// The replica r's ticks by one cluster (tc: thread within the cluster, CT:
// threads of the cluster).  Particle i of the replica stays with thread
// i mod CT for the whole launch (its own writes feed its next MD step);
// nodes, populations and records that other blocks write are read through
// L2.  A replica flagged unstable stops at the next barrier of its cluster.
template <typename T, bool RELAX_FULL>
__device__ __forceinline__ void persistent_replica(const BPersist<T> &q, int r, long long t0, int64_t tc, int64_t CT) {
    using P = Prec<T>;
    using N4 = typename P::node4;
    const BRep<T> &rp = q.l.rep[r];
    if (__ldcg(q.p.unstable + r)) return;
    unsigned long long step = __ldcg(q.l.lb_step + r);
    const int64_t N = (int64_t)rp.nx * rp.ny * rp.nz;
    const int64_t np = rp.np;
    const bool B = rp.variant == LBMD_VARIANT_B;
    const int m = rp.n_sub;
    int cyc = (int)(t0 % (long long)m);
    for (int k = 0; k < q.ticks; ++k) {
        for (int64_t i = tc; i < np; i += CT) batch_couple_particle<T, true>(q.p, rp.part_off + i, r, rp, i, step, cyc);
        const bool due = cyc == m - 1;
        if (B || due) {
            cluster_barrier();
            if (__ldcg(q.p.unstable + r)) break;
        }
        if (B) {
            for (int64_t i = tc; i < np; i += CT) batch_transfer_particle(q.p, rp.part_off + i, rp);
            cluster_barrier();
        }
        if (due) {
            const T *fin = ((step & 1ull) ? q.l.f1 : q.l.f0) + 19 * rp.node_off;
            const N4 *rec = (B ? q.l.node : q.l.jacc) + rp.node_off;
            for (int64_t loc = tc; loc < N; loc += CT) {
                T f[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) f[i] = __ldcg(fin + (int64_t)i * N + loc);
                const N4 n = load_cg(rec + loc);
                batch_collide_node<T, RELAX_FULL>(q.l, rp, step, loc, f, n);
            }
            cluster_barrier();
            const T *fst = ((step & 1ull) ? q.l.f0 : q.l.f1) + 19 * rp.node_off;
            for (int64_t loc = tc; loc < N; loc += CT) {
                T fl[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) fl[i] = __ldcg(fst + (int64_t)i * N + loc);
                batch_moments_node(q.l, rp, loc, fl);
            }
            ++step;
            cluster_barrier();
        }
        cyc = cyc + 1 == m ? 0 : cyc + 1;
    }
    if (tc == 0) q.l.lb_step[r] = step;
}

constexpr int BATCH_PERSIST_THREADS = 256;

template <typename T, bool RELAX_FULL>
__global__ void __launch_bounds__(BATCH_PERSIST_THREADS, sizeof(T) == 4 ? 4 : 2)
    batch_persistent_kernel(BPersist<T> q) {
    const unsigned C = (unsigned)q.cluster;
    const int rank = (int)(blockIdx.x % C), cid = (int)(blockIdx.x / C);
    const int n_clusters = (int)(gridDim.x / C);
    const int64_t tc = (int64_t)rank * blockDim.x + threadIdx.x;
    const int64_t CT = (int64_t)C * blockDim.x;
    const long long t0 = *q.tick0;
    for (int it = 0;; ++it) {
        int32_t *slot = q.taken + 2 * cid + (it & 1);
        if (tc == 0) *slot = (int32_t)atomicAdd(&q.queue[0], 1u);
        cluster_barrier();
        // the slot is written again two iterations on, after every thread of
        // the cluster has passed the next barrier (and so read it)
        const int qi = __ldcg(slot);
        if (qi >= q.R) break;
        persistent_replica<T, RELAX_FULL>(q, q.order[qi], t0, tc, CT);
    }
    if (tc == 0) {
        __threadfence();
        if (atomicAdd(&q.queue[1], 1u) == (unsigned)n_clusters - 1u) *q.tick0 = t0 + q.ticks;
    }
}

template <typename T>
__global__ void batch_init_kernel(T *f, const BRep<T> *rep, int R, int64_t n_total, T rho0) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_total) return;
    // replica of global node g: binary search over node_off
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rep[mid].node_off <= g) lo = mid;
        else hi = mid - 1;
    }
    const BRep<T> &rp = rep[lo];
    const int64_t N = (int64_t)rp.nx * rp.ny * rp.nz, loc = g - rp.node_off;
    T *fr = f + 19 * rp.node_off;
#pragma unroll
    for (int i = 0; i < Q; ++i) fr[(int64_t)i * N + loc] = T(WEIGHT(i)) * rho0;
}

// Per replica: sum of m v^2, of m v (3) and the particle count, FP64 in a
// fixed order (one block per replica).
template <typename T>
__global__ void __launch_bounds__(256) batch_kinetic_kernel(const BRep<T> *rep, const typename Prec<T>::real4 *vel4,
                                                            double *out) {
    __shared__ double sh[4][256];
    const int r = blockIdx.x;
    const BRep<T> &rp = rep[r];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < rp.np; i += blockDim.x) {
        const typename Prec<T>::real4 V = vel4[rp.part_off + i];
        const double m = 1.0 / (double)V.w;
        const double vx = V.x, vy = V.y, vz = V.z;
        v[0] += m * (vx * vx + vy * vy + vz * vz);
        v[1] += m * vx;
        v[2] += m * vy;
        v[3] += m * vz;
    }
    for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[5 * r + threadIdx.x] = sh[threadIdx.x][0];
    if (threadIdx.x == 4) out[5 * r + 4] = (double)rp.np;
}

// FP32 velocities: the sums as FP32 pairs (the FP64 pipes issue far fewer
// operations than the FP32 ones), output order sum m v^2, sum m v
template <>
__global__ void __launch_bounds__(256) batch_kinetic_kernel<float>(const BRep<float> *rep, const float4 *vel4,
                                                                   double *out) {
    const int r = blockIdx.x;
    const BRep<float> &rp = rep[r];
    FF s[4];
    for (int i = threadIdx.x; i < rp.np; i += blockDim.x) {
        const float4 V = vel4[rp.part_off + i];
        add_particle_moments(s, V.x, V.y, V.z, V.w);
    }
    double v[4];
    ff_block_sum<256, 4>(s, v);
    if (threadIdx.x == 0) {
        out[5 * r + 0] = v[3];
        out[5 * r + 1] = v[0];
        out[5 * r + 2] = v[1];
        out[5 * r + 3] = v[2];
        out[5 * r + 4] = (double)rp.np;
    }
}

template <typename T>
__global__ void batch_particles_from_double(const BRep<T> *rep, int r, int64_t first, int64_t count,
                                            typename Prec<T>::real4 *pos4, typename Prec<T>::real4 *vel4,
                                            const double *pos, const double *vel, const double *mass) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const BRep<T> &rp = rep[r];
    const int64_t p = rp.part_off + first + t;
    pos4[p] = pos_from_double<T>(pos + 3 * t, rp.nx, rp.ny, rp.nz);
    vel4[p] = Prec<T>::make4((T)vel[3 * t], (T)vel[3 * t + 1], (T)vel[3 * t + 2], (T)(1.0 / (mass ? mass[t] : 1.0)));
}

template <typename T>
__global__ void batch_particles_to_double(const BRep<T> *rep, int r, const typename Prec<T>::real4 *pos4,
                                          const typename Prec<T>::real4 *vel4, double *pos, double *vel) {
    const BRep<T> &rp = rep[r];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rp.np) return;
    const int64_t p = rp.part_off + i;
    const typename Prec<T>::real4 R = pos4[p], V = vel4[p];
    const CellXYZ c = cell_xyz(Prec<T>::cell_of(R), rp.fd_nx, rp.fd_ny);
    pos[3 * i + 0] = (double)c.x + (double)R.x;
    pos[3 * i + 1] = (double)c.y + (double)R.y;
    pos[3 * i + 2] = (double)c.z + (double)R.z;
    vel[3 * i + 0] = (double)V.x;
    vel[3 * i + 1] = (double)V.y;
    vel[3 * i + 2] = (double)V.z;
}

template <typename T>
__global__ void batch_pops_convert(T *f, int64_t first, int64_t count, double *dst, const double *src) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    if (dst) dst[t] = (double)f[first + t];
    else f[first + t] = (T)src[t];
}

}  // namespace lbmd

using namespace lbmd;

struct lbmd_batch {
    int R = 0;
    int precision = LBMD_FP32;
    std::vector<int> nx, ny, nz, n_sub, variant, cap, np;
    std::vector<double> zeta;
    std::vector<uint64_t> seed;
    std::vector<int64_t> node_off, part_off;
    double rho0 = 1, nu = 1.0 / 6.0, nu_bulk = -1, gamma_ghost = 0, kT = 0;
    FixUnit fix{};  // fixed-point unit of the momentum density (from rho0)
    int64_t n_nodes = 0, n_slots = 0;
    int64_t period = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    LbCoeffs co{};
    // device
    void *f[2] = {nullptr, nullptr};
    void *node = nullptr, *jacc = nullptr;
    void *pos4 = nullptr, *vel4 = nullptr, *fc4 = nullptr, *old4 = nullptr;
    int32_t *prep = nullptr;
    void *rep = nullptr;
    unsigned long long *lb_step = nullptr;
    int *unstable = nullptr;
    unsigned *items_done = nullptr;
    double *kin = nullptr;
    double *staging = nullptr;
    int64_t staging_len = 0;
    // schedule: per tick of the period, the work table (replica, first node)
    // of the due replicas
    int nodes_per_block = 128, particle_block = 256;
    int sms = 1;
    int lb_grid_cap = 0;  // 0: persistent LB grid as large as fits
    bool particles_tuned = false;
    int2 *work = nullptr;
    std::vector<int64_t> work_off, work_len;
    int64_t ticks = 0;  // MD steps done by every replica
    cudaGraphExec_t graph = nullptr;
    double tune_ms_lb[3] = {0, 0, 0}, tune_ms_part[3] = {0, 0, 0};
    // persistent schedule: replicas heaviest first, queue counters, the
    // clusters' taken slots, the device copy of the tick count; graph of one
    // launch for pticks MD steps
    int schedule = LBMD_BATCH_PERIOD_GRAPH;
    int cluster_req = 0;    // blocks per cluster asked for (0: the tuned size)
    int cluster_tuned = 4;  // the autotuner's choice
    double tune_ms_cluster[5] = {0, 0, 0, 0, 0};
    int32_t *order = nullptr;
    unsigned *queue = nullptr;
    int32_t *taken = nullptr;
    int64_t taken_cap = 0;  // clusters the taken array has room for
    long long *dtick = nullptr;
    bool dtick_valid = true;  // the device copy equals ticks
    cudaGraphExec_t pgraph = nullptr;
    int64_t pgraph_ticks = 0;
    int pgraph_cluster = 0;
    std::string err;
};

namespace {

std::mutex g_batch_err_mutex;
std::string g_batch_create_error;

lbmd_status bfail(lbmd_batch *b, lbmd_status s, const std::string &msg) {
    if (b) {
        b->err = msg;
    } else {
        std::lock_guard<std::mutex> lock(g_batch_err_mutex);
        g_batch_create_error = msg;
    }
    return s;
}

lbmd_status bcuda(lbmd_batch *b, cudaError_t e, const char *what) {
    return bfail(b, e == cudaErrorMemoryAllocation ? LBMD_ERR_OOM : LBMD_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define BCK(b, call)                                   \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return bcuda(b, e_, #call); \
    } while (0)

size_t real_bytes(const lbmd_batch *b) { return b->precision == LBMD_FP64 ? 8 : 4; }

void free_batch(lbmd_batch *b) {
    void *bufs[] = {b->f[0], b->f[1],  b->node,  b->jacc,  b->pos4,  b->vel4,  b->fc4,  b->old4,
                    b->prep, b->rep,   b->lb_step, b->unstable, b->items_done, b->kin, b->staging, b->work,
                    b->order, b->queue, b->taken, b->dtick};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->pgraph) cudaGraphExecDestroy(b->pgraph);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

template <typename T>
void fill_reps(const lbmd_batch *b, std::vector<BRep<T>> &out) {
    out.resize(b->R);
    for (int r = 0; r < b->R; ++r) {
        BRep<T> &q = out[r];
        q.nx = b->nx[r];
        q.ny = b->ny[r];
        q.nz = b->nz[r];
        q.n_sub = b->n_sub[r];
        q.variant = b->variant[r];
        q.np = b->np[r];
        q.node_off = b->node_off[r];
        q.part_off = b->part_off[r];
        q.fd_nx = make_fastdiv((uint32_t)b->nx[r]);
        q.fd_ny = make_fastdiv((uint32_t)b->ny[r]);
        q.key0 = (uint32_t)(b->seed[r] & 0xffffffffu);
        q.key1 = (uint32_t)(b->seed[r] >> 32);
        const double dt = 1.0 / (double)b->n_sub[r];
        q.zeta = (T)b->zeta[r];
        q.dt = (T)dt;
        q.half_dt = (T)(0.5 * dt);
        q.amp = (T)std::sqrt(2.0 * b->zeta[r] * b->kT / dt);
        q.neg_scale_dt = (T)dt * -(T)b->fix.scale;
    }
}

template <typename T>
cudaError_t upload_reps(lbmd_batch *b) {
    std::vector<BRep<T>> h;
    fill_reps<T>(b, h);
    return cudaMemcpyAsync(b->rep, h.data(), h.size() * sizeof(BRep<T>), cudaMemcpyHostToDevice, b->stream);
}

// work tables of every tick of the period for the current nodes per item;
// tick k: replicas with (k + 1) % m_r == 0.  "all" table (index period) for
// the initial moments and for tuning.
cudaError_t build_tables(lbmd_batch *b) {
    std::vector<int2> work;
    b->work_off.assign(b->period + 1, 0);
    b->work_len.assign(b->period + 1, 0);
    const int nb = b->nodes_per_block;
    for (int64_t k = 0; k <= b->period; ++k) {
        b->work_off[k] = (int64_t)work.size();
        for (int r = 0; r < b->R; ++r) {
            const bool is_due = k == b->period || (k + 1) % b->n_sub[r] == 0;
            if (!is_due) continue;
            const int64_t N = (int64_t)b->nx[r] * b->ny[r] * b->nz[r];
            for (int64_t s = 0; s < N; s += nb) work.push_back(make_int2(r, (int)s));
        }
        b->work_len[k] = (int64_t)work.size() - b->work_off[k];
    }
    if (b->work) cudaFree(b->work);
    b->work = nullptr;
    cudaError_t e = cudaMalloc(&b->work, std::max<size_t>(1, work.size()) * sizeof(int2));
    if (e != cudaSuccess) return e;
    if (!work.empty()) e = cudaMemcpy(b->work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice);
    return e;
}

template <typename T>
BArgs<T> make_bargs(lbmd_batch *b, int tick) {
    using P = Prec<T>;
    BArgs<T> a;
    a.rep = static_cast<const BRep<T> *>(b->rep);
    a.prep = b->prep;
    a.n_slots = b->n_slots;
    a.pos4 = static_cast<typename P::real4 *>(b->pos4);
    a.vel4 = static_cast<typename P::real4 *>(b->vel4);
    a.fc4 = static_cast<typename P::real4 *>(b->fc4);
    a.old4 = static_cast<typename P::real4 *>(b->old4);
    a.node = static_cast<typename P::node4 *>(b->node);
    a.jacc = static_cast<typename P::node4 *>(b->jacc);
    a.lb_step = b->lb_step;
    a.unstable = b->unstable;
    a.tick = tick;
    a.fis = (T)b->fix.inv_scale;
    return a;
}

template <typename T>
BLbArgs<T> make_lbargs(lbmd_batch *b, int64_t table) {
    BLbArgs<T> a;
    a.rep = static_cast<const BRep<T> *>(b->rep);
    a.work = b->work + b->work_off[table];
    a.n_items = b->work_len[table];
    a.f0 = static_cast<T *>(b->f[0]);
    a.f1 = static_cast<T *>(b->f[1]);
    a.node = static_cast<typename Prec<T>::node4 *>(b->node);
    a.jacc = static_cast<typename Prec<T>::node4 *>(b->jacc);
    a.lb_step = b->lb_step;
    a.unstable = b->unstable;
    a.items_done = b->items_done;
    a.advance = 0;
    a.nodes_per_block = b->nodes_per_block;
    a.fs = (T)b->fix.scale;
    a.fis = (T)b->fix.inv_scale;
    a.gamma_bulk = (T)b->co.gamma_bulk;
    a.gamma_shear = (T)b->co.gamma_shear;
    a.gamma_ghost = (T)b->co.gamma_ghost;
    for (int k = 0; k < Q; ++k) a.amp16[k] = (T)(b->co.noise_amp[k] * 3.4641016151377544 * 1.52587890625e-05);
    a.noisy = b->co.noisy;
    return a;
}

// threads of an LB block: the nodes of one item plus the prefetch warp
int lb_threads(int nodes_per_block) { return nodes_per_block + 32; }

// persistent grid: as many blocks as fit on the GPU at once, at most one per
// item (the kernel's dynamic shared memory allowance is raised to smem first)
template <typename K>
unsigned lb_grid(const lbmd_batch *b, K kernel, int64_t n_items, size_t smem) {
    int per_sm = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, lb_threads(b->nodes_per_block), smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t g = std::min<int64_t>(n_items, (int64_t)per_sm * b->sms);
    if (b->lb_grid_cap > 0) g = std::min<int64_t>(g, b->lb_grid_cap);
    return (unsigned)g;
}

template <typename T>
cudaError_t launch_moments(lbmd_batch *b, const BLbArgs<T> &a) {
    if (a.n_items == 0) return cudaSuccess;
    const size_t smem = lb_smem_bytes<T>(b->nodes_per_block, false);
    batch_moments_kernel<T><<<lb_grid(b, batch_moments_kernel<T>, a.n_items, smem), lb_threads(b->nodes_per_block),
                              smem, b->stream>>>(a);
    return cudaGetLastError();
}

// collide and moments of the work table; with step, the moments kernel
// advances the LB step counters of the replicas it covered
template <typename T>
cudaError_t launch_lb_tables(lbmd_batch *b, int64_t table, bool step) {
    BLbArgs<T> a = make_lbargs<T>(b, table);
    if (a.n_items == 0) return cudaSuccess;
    const int th = lb_threads(b->nodes_per_block);
    const size_t smem = lb_smem_bytes<T>(b->nodes_per_block, true);
    if (b->co.gamma_bulk == 0.0 && b->co.gamma_ghost == 0.0)
        batch_collide_kernel<T, true>
            <<<lb_grid(b, batch_collide_kernel<T, true>, a.n_items, smem), th, smem, b->stream>>>(a);
    else
        batch_collide_kernel<T, false>
            <<<lb_grid(b, batch_collide_kernel<T, false>, a.n_items, smem), th, smem, b->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    a.advance = step ? 1 : 0;
    return launch_moments<T>(b, a);
}

template <typename T>
cudaError_t launch_particles(lbmd_batch *b, const BArgs<T> &a, bool any_b) {
    if (b->n_slots == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((b->n_slots + b->particle_block - 1) / b->particle_block);
    batch_couple_kernel<T><<<blocks, b->particle_block, 0, b->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !any_b) return e;
    batch_transfer_kernel<T><<<blocks, b->particle_block, 0, b->stream>>>(a);
    return cudaGetLastError();
}

bool any_variant_b(const lbmd_batch *b) {
    for (int r = 0; r < b->R; ++r)
        if (b->variant[r] == LBMD_VARIANT_B) return true;
    return false;
}

// one MD tick: all particles, then the LB steps that are due
template <typename T>
cudaError_t launch_tick(lbmd_batch *b, int64_t k) {
    cudaError_t e = launch_particles<T>(b, make_bargs<T>(b, (int)k), any_variant_b(b));
    if (e != cudaSuccess) return e;
    return launch_lb_tables<T>(b, k, true);
}

// Persistent schedule: replicas by estimated work per MD step, heaviest
// first (node updates N / m, the particles, and a fixed share for a tick's
// barriers and latencies), so that the last clusters to start hold the
// lightest replicas.
cudaError_t upload_order(lbmd_batch *b) {
    std::vector<int32_t> o((size_t)b->R);
    std::iota(o.begin(), o.end(), 0);
    std::vector<double> w((size_t)b->R);
    for (int r = 0; r < b->R; ++r)
        w[(size_t)r] = (double)b->nx[r] * b->ny[r] * b->nz[r] / b->n_sub[r] + 8.0 * b->np[r] + 2048.0;
    std::stable_sort(o.begin(), o.end(), [&](int32_t x, int32_t y) { return w[(size_t)x] > w[(size_t)y]; });
    return cudaMemcpyAsync(b->order, o.data(), o.size() * sizeof(int32_t), cudaMemcpyHostToDevice, b->stream);
}

template <typename T>
void persistent_config(lbmd_batch *b, int C, cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at) {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(BATCH_PERSIST_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
}

bool relax_full(const lbmd_batch *b) { return b->co.gamma_bulk == 0.0 && b->co.gamma_ghost == 0.0; }

// clusters of C blocks that fit on the device at once, at most one per
// replica and the taken array's capacity (0: C does not fit)
template <typename T>
int persistent_clusters(lbmd_batch *b, int C) {
    if (C > 8) {  // 16 blocks: a non-portable cluster size
        if (cudaFuncSetAttribute(batch_persistent_kernel<T, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess ||
            cudaFuncSetAttribute(batch_persistent_kernel<T, false>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                 1) != cudaSuccess) {
            (void)cudaGetLastError();
            return 0;
        }
    }
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    persistent_config<T>(b, C, cfg, at);
    int n = 0;
    const cudaError_t e = relax_full(b) ? cudaOccupancyMaxActiveClusters(&n, batch_persistent_kernel<T, true>, &cfg)
                                        : cudaOccupancyMaxActiveClusters(&n, batch_persistent_kernel<T, false>, &cfg);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return (int)std::min<int64_t>({(int64_t)n, (int64_t)b->R, b->taken_cap});
}

// one launch of the persistent kernel for `ticks` MD steps (after zeroing
// the queue counters)
template <typename T>
cudaError_t launch_persistent(lbmd_batch *b, int ticks, int C, int n_clusters) {
    BPersist<T> q;
    q.p = make_bargs<T>(b, 0);
    q.l = make_lbargs<T>(b, 0);
    q.order = b->order;
    q.R = b->R;
    q.ticks = ticks;
    q.cluster = C;
    q.tick0 = b->dtick;
    q.queue = b->queue;
    q.taken = b->taken;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    persistent_config<T>(b, C, cfg, at);
    cfg.gridDim = dim3((unsigned)(n_clusters * C));
    cudaError_t e = cudaMemsetAsync(b->queue, 0, 2 * sizeof(unsigned), b->stream);
    if (e != cudaSuccess) return e;
    return relax_full(b) ? cudaLaunchKernelEx(&cfg, batch_persistent_kernel<T, true>, q)
                         : cudaLaunchKernelEx(&cfg, batch_persistent_kernel<T, false>, q);
}

template <typename T>
cudaError_t init_state(lbmd_batch *b) {
    const unsigned blocks = (unsigned)((b->n_nodes + 255) / 256);
    batch_init_kernel<T><<<blocks, 256, 0, b->stream>>>(static_cast<T *>(b->f[0]), static_cast<BRep<T> *>(b->rep),
                                                         b->R, b->n_nodes, (T)b->rho0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->lb_step, 0, b->R * sizeof(unsigned long long), b->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->dtick, 0, sizeof(long long), b->stream)) != cudaSuccess) return e;
    b->dtick_valid = b->ticks == 0;
    if ((e = cudaMemsetAsync(b->unstable, 0, b->R * sizeof(int), b->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->jacc, 0, b->n_nodes * 4 * real_bytes(b), b->stream)) != cudaSuccess) return e;
    // node field of the rest state: the moments kernel reads buffer
    // (lb_step + 1) & 1, so run it on the "all" table with lb_step = 0 after
    // copying f[0] into f[1]
    if ((e = cudaMemcpyAsync(b->f[1], b->f[0], (size_t)19 * b->n_nodes * real_bytes(b), cudaMemcpyDeviceToDevice,
                             b->stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(b->items_done, 0, b->R * sizeof(unsigned), b->stream)) != cudaSuccess) return e;
    return launch_moments<T>(b, make_lbargs<T>(b, b->period));
}

double time_ms(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    float ms = 0.f;
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    (void)s;
    return (double)ms;
}

// Node kernels: time collide + moments over every replica for each candidate
// block size (on the rest state; the state is re-initialised afterwards).
template <typename T>
cudaError_t tune_lb(lbmd_batch *b) {
    const int cand[3] = {64, 128, 256};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    int best_nb = 128;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
        b->nodes_per_block = cand[c];
        if ((e = build_tables(b)) != cudaSuccess) break;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = launch_lb_tables<T>(b, b->period, false);
        cudaEventRecord(e0, b->stream);
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) e = launch_lb_tables<T>(b, b->period, false);
        cudaEventRecord(e1, b->stream);
        const double ms = time_ms(b->stream, e0, e1) / 3.0;
        b->tune_ms_lb[c] = ms;
        if (ms < best) {
            best = ms;
            best_nb = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    b->nodes_per_block = best_nb;
    return build_tables(b);
}

// Particle kernels: time one tick's particle kernels for each candidate
// block size on copies of the particle state and the node arrays.
template <typename T>
cudaError_t tune_particles(lbmd_batch *b) {
    if (b->n_slots == 0) return cudaSuccess;
    const size_t rs = real_bytes(b);
    const size_t pbytes = (size_t)b->n_slots * 4 * rs, nbytes = (size_t)b->n_nodes * 4 * rs;
    void *pos = nullptr, *vel = nullptr, *fc = nullptr, *old = nullptr, *node = nullptr, *jacc = nullptr;
    int *unst = nullptr;
    cudaError_t e = cudaMalloc(&pos, pbytes);
    if (e == cudaSuccess) e = cudaMalloc(&vel, pbytes);
    if (e == cudaSuccess) e = cudaMalloc(&fc, pbytes);
    if (e == cudaSuccess) e = cudaMalloc(&old, pbytes);
    if (e == cudaSuccess) e = cudaMalloc(&node, nbytes);
    if (e == cudaSuccess) e = cudaMalloc(&jacc, nbytes);
    if (e == cudaSuccess) e = cudaMalloc(&unst, b->R * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(pos, b->pos4, pbytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vel, b->vel4, pbytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(node, b->node, nbytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(jacc, b->jacc, nbytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(unst, b->unstable, b->R * sizeof(int), cudaMemcpyDeviceToDevice, b->stream);
    const int cand[3] = {64, 128, 256};
    if (e == cudaSuccess) {
        BArgs<T> a = make_bargs<T>(b, 0);
        a.pos4 = static_cast<typename Prec<T>::real4 *>(pos);
        a.vel4 = static_cast<typename Prec<T>::real4 *>(vel);
        a.fc4 = static_cast<typename Prec<T>::real4 *>(fc);
        a.old4 = static_cast<typename Prec<T>::real4 *>(old);
        a.node = static_cast<typename Prec<T>::node4 *>(node);
        a.jacc = static_cast<typename Prec<T>::node4 *>(jacc);
        a.unstable = unst;
        const bool anyb = any_variant_b(b);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        double best = 1e300;
        int best_pb = 256;
        for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
            b->particle_block = cand[c];
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = launch_particles<T>(b, a, anyb);
            cudaEventRecord(e0, b->stream);
            for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) e = launch_particles<T>(b, a, anyb);
            cudaEventRecord(e1, b->stream);
            const double ms = time_ms(b->stream, e0, e1) / 5.0;
            b->tune_ms_part[c] = ms;
            if (ms < best) {
                best = ms;
                best_pb = cand[c];
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->particle_block = best_pb;
    }
    cudaStreamSynchronize(b->stream);
    void *bufs[] = {pos, vel, fc, old, node, jacc, unst};
    for (void *p : bufs)
        if (p) cudaFree(p);
    b->particles_tuned = e == cudaSuccess;
    return e;
}

// Persistent schedule: time one period on the current state for each
// cluster size (1, 2, 4, 8 blocks); the state is re-initialised afterwards
// by the caller.
template <typename T>
cudaError_t tune_persistent(lbmd_batch *b) {
    const int cand[5] = {1, 2, 4, 8, 16};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    int best_c = 4;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < 5 && e == cudaSuccess; ++c) {
        b->tune_ms_cluster[c] = 0.0;
        const int nc = persistent_clusters<T>(b, cand[c]);
        if (nc < 1) continue;
        const int k = (int)b->period;
        e = launch_persistent<T>(b, k, cand[c], nc);
        cudaEventRecord(e0, b->stream);
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = launch_persistent<T>(b, k, cand[c], nc);
        cudaEventRecord(e1, b->stream);
        if (e != cudaSuccess) break;
        const double ms = time_ms(b->stream, e0, e1) / 2.0;
        b->tune_ms_cluster[c] = ms;
        if (ms < best) {
            best = ms;
            best_c = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cluster_tuned = best_c;
    return e;
}

// lbmd_batch_run with the persistent schedule: one graph-replayed launch per
// call (a graph per distinct md_steps; the launch reads its first tick from
// the device copy of the tick count, which its last cluster advances)
template <typename T>
lbmd_status run_persistent(lbmd_batch *b, int64_t md_steps) {
    const int C = b->cluster_req ? b->cluster_req : b->cluster_tuned;
    const int nc = persistent_clusters<T>(b, C);
    if (nc < 1) return bfail(b, LBMD_ERR_CUDA, "no cluster of the persistent schedule fits on the device");
    if (!b->dtick_valid) {
        const long long t = b->ticks;
        BCK(b, cudaStreamSynchronize(b->stream));
        BCK(b, cudaMemcpy(b->dtick, &t, sizeof(t), cudaMemcpyHostToDevice));
        b->dtick_valid = true;
    }
    while (md_steps > 0) {
        const int k = (int)std::min<int64_t>(md_steps, (int64_t)1 << 30);
        if (!b->pgraph || b->pgraph_ticks != k || b->pgraph_cluster != C) {
            if (b->pgraph) cudaGraphExecDestroy(b->pgraph);
            b->pgraph = nullptr;
            cudaGraph_t g = nullptr;
            BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            const cudaError_t e = launch_persistent<T>(b, k, C, nc);
            const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return bcuda(b, e, "persistent launch capture");
            }
            if (e2 != cudaSuccess) return bcuda(b, e2, "cudaStreamEndCapture");
            const cudaError_t e3 = cudaGraphInstantiate(&b->pgraph, g, 0);
            cudaGraphDestroy(g);
            if (e3 != cudaSuccess) {
                b->pgraph = nullptr;
                return bcuda(b, e3, "cudaGraphInstantiate");
            }
            b->pgraph_ticks = k;
            b->pgraph_cluster = C;
        }
        BCK(b, cudaGraphLaunch(b->pgraph, b->stream));
        b->ticks += k;
        md_steps -= k;
    }
    return LBMD_OK;
}

#define LBMD_BATCH_DISPATCH(b, FN, ...) \
    ((b)->precision == LBMD_FP64 ? FN<double>(__VA_ARGS__) : FN<float>(__VA_ARGS__))

bool finite_d(double x) { return std::isfinite(x); }

}  // namespace

extern "C" {

const char *lbmd_batch_last_error(lbmd_batch *b) {
    if (b) return b->err.c_str();
    std::lock_guard<std::mutex> lock(g_batch_err_mutex);
    return g_batch_create_error.c_str();
}

lbmd_status lbmd_batch_create(const lbmd_batch_params *p, lbmd_batch **out) {
    if (!p || !out) return bfail(nullptr, LBMD_ERR_ARG, "null argument");
    *out = nullptr;
    const int R = p->n_replicas;
    if (R < 1 || !p->dims || !p->n_sub || !p->variant || !p->zeta || !p->seed || !p->max_particles)
        return bfail(nullptr, LBMD_ERR_ARG, "n_replicas >= 1 and every per-replica array are required");
    if (p->precision != LBMD_FP32 && p->precision != LBMD_FP64)
        return bfail(nullptr, LBMD_ERR_ARG, "batched replicas support LBMD_FP32 and LBMD_FP64");
    if (!(p->rho0 > 0) || !(p->nu > 0) || !finite_d(p->rho0) || !finite_d(p->nu))
        return bfail(nullptr, LBMD_ERR_ARG, "rho0 and nu must be positive");
    if (!(p->kT >= 0) || !finite_d(p->kT)) return bfail(nullptr, LBMD_ERR_ARG, "kT must be >= 0");
    if (!(std::fabs(p->gamma_ghost) < 1.0)) return bfail(nullptr, LBMD_ERR_ARG, "|gamma_ghost| must be < 1");
    lbmd_batch *b = new (std::nothrow) lbmd_batch();
    if (!b) return bfail(nullptr, LBMD_ERR_OOM, "host allocation");
    b->R = R;
    b->precision = p->precision;
    if (!fix_unit(p->rho0, p->precision == LBMD_FP64 ? Prec<double>::SCALE_LOG2 : Prec<float>::SCALE_LOG2, b->fix)) {
        delete b;
        return bfail(nullptr, LBMD_ERR_ARG, "rho0 must lie in [2^-60, 2^60]");
    }
    b->rho0 = p->rho0;
    b->nu = p->nu;
    b->nu_bulk = p->nu_bulk;
    b->gamma_ghost = p->gamma_ghost;
    b->kT = p->kT;
    int64_t nodes = 0, slots = 0, period = 1;
    for (int r = 0; r < R; ++r) {
        const int nx = p->dims[3 * r], ny = p->dims[3 * r + 1], nz = p->dims[3 * r + 2];
        if (nx < 2 || ny < 2 || nz < 2 || nx > BATCH_MAX_EDGE || ny > BATCH_MAX_EDGE || nz > BATCH_MAX_EDGE) {
            delete b;
            return bfail(nullptr, LBMD_ERR_ARG, "replica sides must be in [2, 512]");
        }
        if (p->n_sub[r] < 1 || (p->variant[r] != LBMD_VARIANT_A && p->variant[r] != LBMD_VARIANT_B) ||
            !(p->zeta[r] >= 0) || !finite_d(p->zeta[r]) || p->max_particles[r] < 0) {
            delete b;
            return bfail(nullptr, LBMD_ERR_ARG, "bad n_sub, variant, zeta or max_particles of a replica");
        }
        b->nx.push_back(nx);
        b->ny.push_back(ny);
        b->nz.push_back(nz);
        b->n_sub.push_back(p->n_sub[r]);
        b->variant.push_back(p->variant[r]);
        b->zeta.push_back(p->zeta[r]);
        b->seed.push_back(p->seed[r]);
        b->cap.push_back(p->max_particles[r]);
        b->np.push_back(0);
        b->node_off.push_back(nodes);
        b->part_off.push_back(slots);
        nodes += (int64_t)nx * ny * nz;
        slots += p->max_particles[r];
        period = std::lcm(period, (int64_t)p->n_sub[r]);
        if (period > BATCH_MAX_PERIOD) {
            delete b;
            return bfail(nullptr, LBMD_ERR_ARG, "the lcm of the replicas' n_sub must not exceed 256");
        }
    }
    if (nodes > (int64_t)0x7fffffff || slots > (int64_t)0x7fffffff) {
        delete b;
        return bfail(nullptr, LBMD_ERR_ARG, "more than 2^31-1 nodes or particle slots in the batch");
    }
    b->n_nodes = nodes;
    b->n_slots = slots;
    b->period = period;
    // relaxation factors and noise amplitudes, as for a single box
    lb_coefficients(p->nu, p->nu_bulk, p->gamma_ghost, p->kT, b->co);
    if (p->stream) {
        b->stream = (cudaStream_t)p->stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            lbmd_status s = bcuda(nullptr, e, "cudaStreamCreate");
            delete b;
            return s;
        }
        b->own_stream = true;
    }
    const size_t rs = real_bytes(b);
    const int64_t sl = std::max<int64_t>(1, slots);
    b->staging_len = std::max<int64_t>((int64_t)1 << 20, 19 * 512 * 512);
    struct {
        void **ptr;
        size_t bytes;
    } allocs[] = {
        {&b->f[0], (size_t)19 * nodes * rs},
        {&b->f[1], (size_t)19 * nodes * rs},
        {&b->node, (size_t)nodes * 4 * rs},
        {&b->jacc, (size_t)nodes * 4 * rs},
        {&b->pos4, (size_t)sl * 4 * rs},
        {&b->vel4, (size_t)sl * 4 * rs},
        {&b->fc4, (size_t)sl * 4 * rs},
        {&b->old4, (size_t)sl * 4 * rs},
        {(void **)&b->prep, (size_t)sl * sizeof(int32_t)},
        {&b->rep, (size_t)R * (b->precision == LBMD_FP64 ? sizeof(BRep<double>) : sizeof(BRep<float>))},
        {(void **)&b->lb_step, (size_t)R * sizeof(unsigned long long)},
        {(void **)&b->unstable, (size_t)R * sizeof(int)},
        {(void **)&b->items_done, (size_t)R * sizeof(unsigned)},
        {(void **)&b->kin, (size_t)R * 5 * sizeof(double)},
        {(void **)&b->staging, (size_t)b->staging_len * sizeof(double)},
        {(void **)&b->order, (size_t)R * sizeof(int32_t)},
        {(void **)&b->queue, 2 * sizeof(unsigned)},
        {(void **)&b->dtick, sizeof(long long)},
    };
    for (auto &a : allocs) {
        cudaError_t e = cudaMalloc(a.ptr, a.bytes);
        if (e != cudaSuccess) {
            lbmd_status s = bcuda(nullptr, e, "cudaMalloc");
            free_batch(b);
            delete b;
            return s;
        }
    }
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
        if (b->sms < 1) b->sms = 1;
        // resident clusters of the persistent schedule: at most 32 blocks per SM
        b->taken_cap = (int64_t)b->sms * 32;
        const cudaError_t e = cudaMalloc(&b->taken, (size_t)2 * b->taken_cap * sizeof(int32_t));
        if (e != cudaSuccess) {
            lbmd_status s = bcuda(nullptr, e, "cudaMalloc");
            free_batch(b);
            delete b;
            return s;
        }
    }
    std::vector<int32_t> prep((size_t)sl, 0);
    for (int r = 0; r < R; ++r)
        for (int64_t i = 0; i < b->cap[r]; ++i) prep[(size_t)(b->part_off[r] + i)] = r;
    cudaError_t e = cudaMemcpy(b->prep, prep.data(), prep.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = LBMD_BATCH_DISPATCH(b, upload_reps, b);
    if (e == cudaSuccess) e = build_tables(b);
    if (e == cudaSuccess) e = LBMD_BATCH_DISPATCH(b, init_state, b);
    if (e == cudaSuccess) e = upload_order(b);
    if (e == cudaSuccess) e = LBMD_BATCH_DISPATCH(b, tune_lb, b);
    if (e == cudaSuccess) e = LBMD_BATCH_DISPATCH(b, tune_persistent, b);
    if (e == cudaSuccess) e = LBMD_BATCH_DISPATCH(b, init_state, b);  // tuning stepped the populations
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        lbmd_status s = bcuda(nullptr, e, "batch initialisation");
        free_batch(b);
        delete b;
        return s;
    }
    *out = b;
    return LBMD_OK;
}

lbmd_status lbmd_batch_destroy(lbmd_batch *b) {
    if (!b) return LBMD_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
    return LBMD_OK;
}

lbmd_status lbmd_batch_add_particles(lbmd_batch *b, int32_t r, int64_t n, const double *pos, const double *vel,
                                     const double *mass) {
    if (!b) return LBMD_ERR_ARG;
    if (r < 0 || r >= b->R || n < 0 || (n > 0 && (!pos || !vel))) return bfail(b, LBMD_ERR_ARG, "bad arguments");
    if (b->np[r] + n > b->cap[r]) return bfail(b, LBMD_ERR_CAPACITY, "replica particle capacity exceeded");
    for (int64_t q = 0; q < 3 * n; ++q)
        if (!finite_d(pos[q]) || !finite_d(vel[q])) return bfail(b, LBMD_ERR_ARG, "non-finite particle data");
    if (mass)
        for (int64_t q = 0; q < n; ++q)
            if (!(mass[q] > 0) || !finite_d(mass[q])) return bfail(b, LBMD_ERR_ARG, "mass must be positive");
    if (n == 0) return LBMD_OK;
    if (7 * n > b->staging_len) return bfail(b, LBMD_ERR_CAPACITY, "too many particles in one call");
    double *dpos = b->staging, *dvel = b->staging + 3 * n, *dm = b->staging + 6 * n;
    BCK(b, cudaMemcpyAsync(dpos, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(dvel, vel, 3 * n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    if (mass) BCK(b, cudaMemcpyAsync(dm, mass, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (b->precision == LBMD_FP64)
        batch_particles_from_double<double><<<blocks, 256, 0, b->stream>>>(
            static_cast<BRep<double> *>(b->rep), r, b->np[r], n, static_cast<D4 *>(b->pos4),
            static_cast<D4 *>(b->vel4), dpos, dvel, mass ? dm : nullptr);
    else
        batch_particles_from_double<float><<<blocks, 256, 0, b->stream>>>(
            static_cast<BRep<float> *>(b->rep), r, b->np[r], n, static_cast<float4 *>(b->pos4),
            static_cast<float4 *>(b->vel4), dpos, dvel, mass ? dm : nullptr);
    BCK(b, cudaGetLastError());
    b->np[r] += (int)n;
    BCK(b, LBMD_BATCH_DISPATCH(b, upload_reps, b));
    BCK(b, upload_order(b));
    BCK(b, cudaStreamSynchronize(b->stream));
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->particles_tuned = false;
    return LBMD_OK;
}

lbmd_status lbmd_batch_run(lbmd_batch *b, int64_t md_steps) {
    LBMD_TRACE("lbmd_batch_run");
    if (!b || md_steps < 0) return LBMD_ERR_ARG;
    if (b->schedule == LBMD_BATCH_PERSISTENT) return LBMD_BATCH_DISPATCH(b, run_persistent, b, md_steps);
    if (!b->particles_tuned && b->n_slots > 0) BCK(b, LBMD_BATCH_DISPATCH(b, tune_particles, b));
    if (md_steps > 0) b->dtick_valid = false;  // the device tick copy serves the persistent schedule only
    int64_t left = md_steps;
    // eager ticks up to the next period boundary, whole periods from the
    // captured graph, eager ticks for the rest
    while (left > 0 && b->ticks % b->period != 0) {
        BCK(b, LBMD_BATCH_DISPATCH(b, launch_tick, b, b->ticks % b->period));
        ++b->ticks;
        --left;
    }
    while (left >= b->period) {
        if (!b->graph) {
            cudaGraph_t g = nullptr;
            BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int64_t k = 0; k < b->period && e == cudaSuccess; ++k) e = LBMD_BATCH_DISPATCH(b, launch_tick, b, k);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return bcuda(b, e, "capture");
            }
            if (e2 != cudaSuccess) return bcuda(b, e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                b->graph = nullptr;
                return bcuda(b, e, "cudaGraphInstantiate");
            }
        }
        BCK(b, cudaGraphLaunch(b->graph, b->stream));
        b->ticks += b->period;
        left -= b->period;
    }
    while (left > 0) {
        BCK(b, LBMD_BATCH_DISPATCH(b, launch_tick, b, b->ticks % b->period));
        ++b->ticks;
        --left;
    }
    return LBMD_OK;
}

lbmd_status lbmd_batch_kinetic_device(lbmd_batch *b, double *out) {
    if (!b || !out) return LBMD_ERR_ARG;
    if (b->precision == LBMD_FP64)
        batch_kinetic_kernel<double><<<b->R, 256, 0, b->stream>>>(static_cast<BRep<double> *>(b->rep),
                                                                   static_cast<D4 *>(b->vel4), out);
    else
        batch_kinetic_kernel<float><<<b->R, 256, 0, b->stream>>>(static_cast<BRep<float> *>(b->rep),
                                                                  static_cast<float4 *>(b->vel4), out);
    BCK(b, cudaGetLastError());
    return LBMD_OK;
}

lbmd_status lbmd_batch_kinetic(lbmd_batch *b, double *out) {
    if (!b || !out) return LBMD_ERR_ARG;
    lbmd_status s = lbmd_batch_kinetic_device(b, b->kin);
    if (s != LBMD_OK) return s;
    BCK(b, cudaMemcpyAsync(out, b->kin, (size_t)b->R * 5 * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return LBMD_OK;
}

lbmd_status lbmd_batch_unstable(lbmd_batch *b, int32_t *out) {
    if (!b || !out) return LBMD_ERR_ARG;
    std::vector<int> h(b->R);
    BCK(b, cudaMemcpyAsync(h.data(), b->unstable, b->R * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    for (int r = 0; r < b->R; ++r) out[r] = h[r];
    return LBMD_OK;
}

lbmd_status lbmd_batch_get_counts(lbmd_batch *b, int32_t r, int64_t *n_particles, int64_t *lb_step,
                                  int64_t *md_step) {
    if (!b || r < 0 || r >= b->R) return LBMD_ERR_ARG;
    unsigned long long s = 0;
    BCK(b, cudaMemcpyAsync(&s, b->lb_step + r, sizeof(s), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    if (n_particles) *n_particles = b->np[r];
    if (lb_step) *lb_step = (int64_t)s;
    if (md_step) *md_step = b->ticks;
    return LBMD_OK;
}

static lbmd_status batch_pops(lbmd_batch *b, int32_t r, double *out, const double *in) {
    if (!b || r < 0 || r >= b->R || (!out && !in)) return LBMD_ERR_ARG;
    unsigned long long s = 0;
    BCK(b, cudaMemcpyAsync(&s, b->lb_step + r, sizeof(s), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    const int64_t N = (int64_t)b->nx[r] * b->ny[r] * b->nz[r], total = 19 * N, base = 19 * b->node_off[r];
    void *fb = b->f[s & 1ull];
    for (int64_t c0 = 0; c0 < total; c0 += b->staging_len) {
        const int64_t c = std::min(b->staging_len, total - c0);
        const unsigned blocks = (unsigned)((c + 255) / 256);
        if (in) BCK(b, cudaMemcpyAsync(b->staging, in + c0, c * sizeof(double), cudaMemcpyHostToDevice, b->stream));
        if (b->precision == LBMD_FP64)
            batch_pops_convert<double><<<blocks, 256, 0, b->stream>>>(static_cast<double *>(fb), base + c0, c,
                                                                      out ? b->staging : nullptr, b->staging);
        else
            batch_pops_convert<float><<<blocks, 256, 0, b->stream>>>(static_cast<float *>(fb), base + c0, c,
                                                                     out ? b->staging : nullptr, b->staging);
        BCK(b, cudaGetLastError());
        if (out) BCK(b, cudaMemcpyAsync(out + c0, b->staging, c * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
    }
    return LBMD_OK;
}

lbmd_status lbmd_batch_get_populations(lbmd_batch *b, int32_t r, double *out) { return batch_pops(b, r, out, nullptr); }

lbmd_status lbmd_batch_set_populations(lbmd_batch *b, int32_t r, const double *in) {
    if (!b || !in || r < 0 || r >= b->R) return LBMD_ERR_ARG;
    // between its LB steps a replica's node field carries transfers
    if (b->ticks % b->n_sub[r] != 0)
        return bfail(b, LBMD_ERR_SEQUENCE, "set_populations only at the replica's cycle boundary");
    lbmd_status s = batch_pops(b, r, nullptr, in);
    if (s != LBMD_OK) return s;
    // node field of the new populations: the moments kernel reads buffer
    // (lb_step + 1) & 1, so mirror the current buffer there first
    unsigned long long st = 0;
    BCK(b, cudaMemcpyAsync(&st, b->lb_step + r, sizeof(st), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    const int64_t N = (int64_t)b->nx[r] * b->ny[r] * b->nz[r];
    const size_t rs = real_bytes(b), off = (size_t)19 * b->node_off[r] * rs;
    BCK(b, cudaMemcpyAsync((char *)b->f[(st + 1) & 1ull] + off, (char *)b->f[st & 1ull] + off, (size_t)19 * N * rs,
                           cudaMemcpyDeviceToDevice, b->stream));
    // a one-replica work table
    std::vector<int2> w;
    for (int64_t s0 = 0; s0 < N; s0 += b->nodes_per_block) w.push_back(make_int2(r, (int)s0));
    int2 *dw = nullptr;
    BCK(b, cudaMalloc(&dw, w.size() * sizeof(int2)));
    cudaError_t e = cudaMemcpy(dw, w.data(), w.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (b->precision == LBMD_FP64) {
            BLbArgs<double> a = make_lbargs<double>(b, 0);
            a.work = dw;
            a.n_items = (int64_t)w.size();
            e = launch_moments<double>(b, a);
        } else {
            BLbArgs<float> a = make_lbargs<float>(b, 0);
            a.work = dw;
            a.n_items = (int64_t)w.size();
            e = launch_moments<float>(b, a);
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync((char *)b->jacc + (size_t)b->node_off[r] * 4 * rs, 0, (size_t)N * 4 * rs,
                                              b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(dw);
    if (e != cudaSuccess) return bcuda(b, e, "set_populations");
    return LBMD_OK;
}

lbmd_status lbmd_batch_get_particles(lbmd_batch *b, int32_t r, double *pos, double *vel) {
    if (!b || r < 0 || r >= b->R || !pos || !vel) return LBMD_ERR_ARG;
    const int64_t n = b->np[r];
    if (n == 0) return LBMD_OK;
    if (6 * n > b->staging_len) return bfail(b, LBMD_ERR_CAPACITY, "staging buffer too small");
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (b->precision == LBMD_FP64)
        batch_particles_to_double<double><<<blocks, 256, 0, b->stream>>>(static_cast<BRep<double> *>(b->rep), r,
                                                                         static_cast<D4 *>(b->pos4),
                                                                         static_cast<D4 *>(b->vel4), b->staging,
                                                                         b->staging + 3 * n);
    else
        batch_particles_to_double<float><<<blocks, 256, 0, b->stream>>>(static_cast<BRep<float> *>(b->rep), r,
                                                                        static_cast<float4 *>(b->pos4),
                                                                        static_cast<float4 *>(b->vel4), b->staging,
                                                                        b->staging + 3 * n);
    BCK(b, cudaGetLastError());
    BCK(b, cudaMemcpyAsync(pos, b->staging, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaMemcpyAsync(vel, b->staging + 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return LBMD_OK;
}

lbmd_status lbmd_batch_tuning(lbmd_batch *b, int32_t *nodes_per_block, int32_t *particle_block, double *lb_ms,
                              double *particle_ms) {
    if (!b) return LBMD_ERR_ARG;
    if (nodes_per_block) *nodes_per_block = b->nodes_per_block;
    if (particle_block) *particle_block = b->particle_block;
    for (int c = 0; c < 3; ++c) {
        if (lb_ms) lb_ms[c] = b->tune_ms_lb[c];
        if (particle_ms) particle_ms[c] = b->tune_ms_part[c];
    }
    return LBMD_OK;
}

lbmd_status lbmd_batch_set_lb_grid(lbmd_batch *b, int32_t max_blocks) {
    if (!b) return LBMD_ERR_ARG;
    if (max_blocks < 0) return bfail(b, LBMD_ERR_ARG, "max_blocks must be >= 0");
    BCK(b, cudaStreamSynchronize(b->stream));
    b->lb_grid_cap = max_blocks;
    if (b->graph) {  // the captured period has the old grid size baked in
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return LBMD_OK;
}

lbmd_status lbmd_batch_set_schedule(lbmd_batch *b, int32_t schedule, int32_t cluster_blocks) {
    if (!b) return LBMD_ERR_ARG;
    if (schedule != LBMD_BATCH_PERIOD_GRAPH && schedule != LBMD_BATCH_PERSISTENT)
        return bfail(b, LBMD_ERR_ARG, "unknown schedule");
    if (cluster_blocks != 0 && cluster_blocks != 1 && cluster_blocks != 2 && cluster_blocks != 4 && cluster_blocks != 8 &&
        cluster_blocks != 16)
        return bfail(b, LBMD_ERR_ARG, "cluster_blocks must be 0, 1, 2, 4, 8 or 16");
    BCK(b, cudaStreamSynchronize(b->stream));
    if (schedule == LBMD_BATCH_PERSISTENT && cluster_blocks != 0 &&
        LBMD_BATCH_DISPATCH(b, persistent_clusters, b, cluster_blocks) < 1)
        return bfail(b, LBMD_ERR_ARG, "a cluster of that many blocks does not fit on the device");
    b->schedule = schedule;
    b->cluster_req = cluster_blocks;
    return LBMD_OK;
}

lbmd_status lbmd_batch_persistent_tuning(lbmd_batch *b, int32_t *cluster_blocks, double *ms) {
    if (!b) return LBMD_ERR_ARG;
    if (cluster_blocks) *cluster_blocks = b->cluster_tuned;
    if (ms)
        for (int c = 0; c < 5; ++c) ms[c] = b->tune_ms_cluster[c];
    return LBMD_OK;
}

void *lbmd_batch_stream(lbmd_batch *b) { return b ? (void *)b->stream : nullptr; }

}  // extern "C"
