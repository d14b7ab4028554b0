// M2L on the tensor cores (tcgen05, sm_103a).
//
// Same-level M2L (Sec. 2.1 of Yokota & Barba, arXiv:1106.2176) is a dense
// contraction once the expansions are scaled by their cell width: for a tile
// of 128 target cells of one level and one octant and a translation vector v
// of the octant's stencil,
//     L~[128 x p^2] += gather_v(M~)[128 x p^2] * T_v^T,
// T_v the level-independent p^2 x p^2 real operator. Sec. 5 notes that M2L at
// all levels needs no synchronisation between levels: one launch covers every
// level's tiles.
//
// Precision: A = M~ and B = T_v are split into two TF32 values each, hi and
// lo (round to nearest), and the MMAs compute A_hi [T_hi ; T_lo] (N = 2 NP)
// plus A_lo T_hi, accumulating in FP32 in tensor memory: the main sum in
// columns [0, NP), the small correction terms in [NP, 2 NP). Every GV vectors
// the accumulator is drained into per-thread FP32 (hi, lo) TwoSum registers;
// two TMEM buffers alternate so the drain overlaps the next MMAs.
//
// Per CTA (128 threads, one per target row), for every unit (v, k-block):
//   - the thread finds its source cell (lattice lookup) and copies its 256 B
//     (hi, lo) row with cp.async into the 128B-swizzled A tiles (zero fill if
//     the cell is absent);
//   - thread 0 bulk-copies the pre-swizzled [T_hi ; T_lo] k-block image and,
//     once all rows of the stage are in, issues the tcgen05.mma and commits to
//     the stage's mbarrier.
// Stages rotate through NS buffers. Every wait is bounded; on a timeout the
// kernel records an error code and leaves after releasing its TMEM.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "fmm_internal.cuh"

namespace fmm {

static inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *b, uint32_t tx)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(b)),
                 "r"(tx)
                 : "memory");
}

// bounded wait for the given phase parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity)
{
    const uint32_t a = smem_u32(b);
    for (int it = 0; it < (1 << 20); it++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 128B-swizzled, K-major shared-memory matrix descriptor (SBO = 1024 B between
// 8-row groups; LBO unused for this layout)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused): 16 B
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: 1024 B
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

// instruction descriptor: D f32, A and B tf32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive TMEM columns of this warp's 32 lanes (one row per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_rn(float a)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
    return __uint_as_float(r);
}

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b)
{
    const float s = hi + b;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}

// ---------------------------------------------------------------------------
// tile geometry
// ---------------------------------------------------------------------------
template <int NP, int KB>
struct TcCfg {
    static constexpr int M = 128;                         // target rows per tile
    static constexpr int A_BYTES = M * 128;               // one k-block of A (hi or lo)
    static constexpr int B_BYTES = 2 * NP * 128;          // one k-block of [T_hi ; T_lo]
    static constexpr int STAGE = 2 * A_BYTES + B_BYTES;   // multiple of 1024
    // three stages at most: the CTA then leaves room on its SM for two P2P
    // blocks, which run concurrently on the other stream and use the FMA pipes
    // this latency-bound kernel leaves idle
    static constexpr int NS = (150 * 1024) / STAGE >= 3 ? 3 : 2;
    static constexpr int QV = 8;                           // lookahead of the source lookups (vectors)
    static constexpr int RING = 2 * QV * M * 4;            // lookup ring: 2 QV slots x 128 rows
    static constexpr int FIXED = NS * STAGE + 256 + RING;  // stages, barriers, lookup ring
    static constexpr int SMEM_MAX = 227 * 1024 - 1024;     // minus the alignment slack
    static constexpr int ST_MAX = 0;                       // stencil read through L1 (keeps shared memory small)
    static constexpr int TCOLS = 4 * NP <= 32 ? 32 : (4 * NP <= 64 ? 64 : (4 * NP <= 128 ? 128 : (4 * NP <= 256 ? 256 : 512)));
    static constexpr int GV = 8;                          // vectors per accumulator drain
    static constexpr bool COMP = NP <= 64;                // compensated registers for the drained sums
};

// Split the scaled multipoles into TF32 (hi, lo) rows: out[c][kb][hi 32 | lo 32].
__global__ void msplit_k(const float *__restrict__ M, int PP, int KB, int c0, int nc, float *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int KP = KB * 32;
    if (i >= (int64_t)(nc - c0) * KP) return;
    const int c = c0 + (int)(i / KP), k = (int)(i % KP);
    const float a = k < PP ? M[(size_t)c * PP + k] : 0.f;
    const float hi = tf32_rn(a);
    const float lo = tf32_rn(a - hi);
    const int kb = k >> 5, kk = k & 31;
    float *o = out + ((size_t)c * KB + kb) * 64;
    o[kk] = hi;
    o[32 + kk] = lo;
}

template <int NP, int KB>
__global__ void __launch_bounds__(128, 1)
    m2l_tc_k(int p, const M2LTile *__restrict__ tiles, const int *__restrict__ ntiles, const int *__restrict__ tgt,
             const int4 *__restrict__ xyz, const uint64_t *__restrict__ anchor, const LevelDesc *__restrict__ ld,
             const int *__restrict__ map_pool, const int4 *__restrict__ st, const int *__restrict__ st_off,
             const float *__restrict__ msplit, const unsigned char *__restrict__ ttab, float *__restrict__ L,
             int *__restrict__ err)
{
    using C = TcCfg<NP, KB>;
    constexpr int NS = C::NS;
    if ((int)blockIdx.x >= *ntiles) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned start for the swizzled tiles (kept as a shared-array offset)
    unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + NS * C::STAGE);
    int *ring = reinterpret_cast<int *>(base + NS * C::STAGE + 256);          // [2 QV][128]
    int4 *s_st = reinterpret_cast<int4 *>(base + NS * C::STAGE + 256 + C::RING); // stencil of the octant
    uint64_t *full_a = bar;            // NS, 128 arrivals
    uint64_t *full_b = bar + NS;       // NS, 1 arrival + tx bytes
    uint64_t *mma_done = bar + 2 * NS; // NS, MMA commits
    uint64_t *acc_full = bar + 3 * NS; // 2, MMA commits
    uint64_t *acc_empty = bar + 3 * NS + 2; // 2, 128 arrivals
    uint64_t *fin = bar + 3 * NS + 4;       // 1, final MMA flush after an abort
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 3 * NS + 5);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5;
    const M2LTile td = tiles[blockIdx.x];
    const int PP = p * p;
    const int l = td.level, sh = FMM_MAXLEVEL - l;
    int px = 0, py = 0, pz = 0, cell = -1;
    if (tid < td.count) {
        cell = tgt[td.start + tid];
        const int4 a = xyz[cell];
        px = a.x >> sh;
        py = a.y >> sh;
        pz = a.z >> sh;
    }
    const LevelDesc LD = ld[l];

    if (tid == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(&full_a[s], 128);
            mbar_init(&full_b[s], 1);
            mbar_init(&mma_done[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int e0 = st_off[td.octant], e1 = st_off[td.octant + 1];
    const int nv = e1 - e0;
    const int nunits = nv * KB;
    const int ngroups = (nv + C::GV - 1) / C::GV;

    // per-thread accumulators of the drained sums (row = tid)
    float acc_hi[NP], acc_lo[C::COMP ? NP : 1];
#pragma unroll
    for (int k = 0; k < NP; k++) acc_hi[k] = 0.f;
#pragma unroll
    for (int k = 0; k < (C::COMP ? NP : 1); k++) acc_lo[k] = 0.f;

    // The stencil of the octant in shared memory when it fits.
    const bool st_in_smem = nv <= C::ST_MAX;
    if (st_in_smem)
        for (int i = tid; i < nv; i += 128) s_st[i] = st[e0 + i];
    __syncthreads();
    const int4 *stp = st_in_smem ? s_st : st + e0;

    // Source cell of vector vi for this row, fetched QV vectors ahead of use
    // into ring slot vi % (2 QV): with a dense lattice map the entry is copied
    // by cp.async straight into shared memory, so no load result is waited
    // for on the critical path; other levels search the level's sorted keys.
    constexpr int QV = C::QV;
    auto fetch = [&](int vi) {
        const uint32_t slot = smem_u32(ring + (vi % (2 * QV)) * 128 + tid);
        int r = -1;
        if (cell >= 0 && vi < nv) {
            const int4 v = stp[vi];
            const int x = px + v.x, y = py + v.y, z = pz + v.z, side = 1 << l;
            if (x >= 0 && y >= 0 && z >= 0 && x < side && y < side && z < side) {
                if (LD.map_off >= 0) {
                    cp_async4(slot, map_pool + LD.map_off + (long long)morton3((uint32_t)x, (uint32_t)y, (uint32_t)z));
                    return;
                }
                r = level_lookup(LD, map_pool, anchor, l, x, y, z);
            }
        }
        ring[(vi % (2 * QV)) * 128 + tid] = r;
    };
    for (int i = 0; i < QV; i++) fetch(i);
    cp_async_commit();
    cp_async_wait_all();
    int src = -1;
    int issued_b = 0;  // thread 0: operator copies issued
    auto load_unit = [&](int u) {
        const int s = u % NS;
        const int vi = u / KB, kb = u % KB;
        if (kb == 0) {
            src = ring[(vi % (2 * QV)) * 128 + tid];
            fetch(vi + QV);
        }
        unsigned char *sa = base + s * C::STAGE;
        const uint32_t ahi = smem_u32(sa), alo = smem_u32(sa + C::A_BYTES);
        // the warp copies its 32 rows: 16 lanes per 256-byte (hi | lo) row, so
        // every instruction reads two whole rows; the source cell of a row
        // comes from the lane that owns it
        const int lane = tid & 31, ch = lane & 15;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int r = 2 * i + (lane >> 4);
            const int sr = __shfl_sync(0xffffffffu, src, r);
            const int row = (warp << 5) + r;
            const float *g = msplit + ((size_t)(sr >= 0 ? sr : 0) * KB + kb) * 64 + ch * 4;
            const uint32_t dst = (ch < 8 ? ahi : alo) + (uint32_t)row * 128u + ((((uint32_t)ch & 7u) ^ ((uint32_t)row & 7u)) << 4);
            cp_async16(dst, g, sr >= 0 ? 16u : 0u);
        }
        cp_async_commit();
        if (tid == 0) {
            const int4 v = stp[vi];
            mbar_arrive_tx(&full_b[s], C::B_BYTES);
            bulk_g2s(smem_u32(sa + 2 * C::A_BYTES), ttab + ((size_t)v.w * KB + kb) * C::B_BYTES, C::B_BYTES, &full_b[s]);
            issued_b = u + 1;
        }
    };

    auto drain = [&](int g) {
        const int b = g & 1;
        __syncwarp();
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], (uint32_t)((g >> 1) & 1)));
        if (!ok) {
            atomicExch(abort_flag, 1);
            return;
        }
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * 2 * NP);
        float mv[16], cv[16];
#pragma unroll
        for (int k0 = 0; k0 < NP; k0 += 16) {
            tmem_ld16(taddr + k0, mv);
            tmem_ld16(taddr + NP + k0, cv);
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const float t = mv[k] + cv[k];
                if (C::COMP) two_sum_acc(acc_hi[k0 + k], acc_lo[C::COMP ? k0 + k : 0], t);
                else acc_hi[k0 + k] += t;
            }
        }
        tc_fence_before();
        mbar_arrive(&acc_empty[b]);
    };

    // prologue: the first NS-1 units in flight
    for (int u = 0; u < NS - 1 && u < nunits; u++) load_unit(u);

    const uint32_t id_full = idesc_tf32(128, 2 * NP), id_half = idesc_tf32(128, NP);
    int drained = 0;
    int consumed = 0;  // thread 0: units whose operator copy has been waited for
    for (int u = 0; u < nunits; u++) {
        if (*(volatile int *)abort_flag) break;
        const int s = u % NS;
        // this thread's rows of unit u have landed
        if (u + NS - 1 <= nunits) cp_async_wait<NS - 2>();
        else cp_async_wait_all();
        fence_proxy_async();
        mbar_arrive(&full_a[s]);
        if (tid == 0) {
            const uint32_t par = (uint32_t)((u / NS) & 1);
            bool ok = mbar_wait(&full_a[s], par) && mbar_wait(&full_b[s], par);
            if (ok) consumed = u + 1;
            const int vi = u / KB, kb = u % KB, g = vi / C::GV;
            const int b = g & 1;
            // first unit of a group: the buffer must have been drained
            if (ok && kb == 0 && vi % C::GV == 0 && g >= 2) ok = mbar_wait(&acc_empty[b], (uint32_t)(((g - 2) >> 1) & 1));
            if (!ok) {
                atomicExch(abort_flag, 1);
            } else {
                fence_proxy_async();
                tc_fence_after();
                unsigned char *sa = base + s * C::STAGE;
                const uint32_t ahi = smem_u32(sa), alo = smem_u32(sa + C::A_BYTES), bb = smem_u32(sa + 2 * C::A_BYTES);
                const uint32_t dmain = tmem + (uint32_t)(b * 2 * NP), dcorr = dmain + NP;
                const bool first = (vi % C::GV == 0) && kb == 0;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    // A_hi [T_hi ; T_lo] -> main | correction, then A_lo T_hi -> correction
                    mma_tf32(dmain, sdesc(ahi + 32 * k), sdesc(bb + 32 * k), id_full, (first && k == 0) ? 0u : 1u);
                    mma_tf32(dcorr, sdesc(alo + 32 * k), sdesc(bb + 32 * k), id_half, 1u);
                }
                mma_commit(&mma_done[s]);
                const bool last_of_group = (kb == KB - 1) && ((vi % C::GV == C::GV - 1) || vi == nv - 1);
                if (last_of_group) mma_commit(&acc_full[b]);
            }
        }
        // refill: unit u + NS - 1 reuses the stage of unit u - 1
        const int un = u + NS - 1;
        if (un < nunits) {
            if (u >= 1 && !mbar_wait(&mma_done[(u - 1) % NS], (uint32_t)(((u - 1) / NS) & 1))) {
                atomicExch(abort_flag, 1);
                break;
            }
            load_unit(un);
        }
        // drain group g - 1 once group g is well under way
        const int vi = u / KB;
        if ((u % KB) == KB - 1 && vi % C::GV == 2 && vi / C::GV >= 1 && drained < vi / C::GV) {
            drain(drained);
            drained++;
        }
    }
    cp_async_wait_all();
    if (tid == 0 && *(volatile int *)abort_flag) {
        // wait (bounded) for the operator copies still in flight and the MMAs
        for (int u = consumed; u < issued_b; u++) mbar_wait(&full_b[u % NS], (uint32_t)((u / NS) & 1));
        mma_commit(fin);
        mbar_wait(fin, 0);
    }
    __syncthreads();
    if (!*(volatile int *)abort_flag) {
        while (drained < ngroups) {
            drain(drained);
            drained++;
            if (*(volatile int *)abort_flag) break;
        }
    }
    // every MMA commit must have arrived before the shared memory goes away
    if (tid == 0 && !*(volatile int *)abort_flag)
        for (int u = max(0, nunits - NS); u < nunits; u++) mbar_wait(&mma_done[u % NS], (uint32_t)((u / NS) & 1));
    if (cell >= 0 && !*(volatile int *)abort_flag) {
        float *Lc = L + (size_t)cell * PP;
#pragma unroll
        for (int k = 0; k < NP; k++)
            if (k < PP) Lc[k] += C::COMP ? acc_hi[k] + acc_lo[C::COMP ? k : 0] : acc_hi[k];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TCOLS));
    }
    if (tid == 0 && *(volatile int *)abort_flag) atomicExch(err, 1);
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
struct TcShape {
    int NP, KB;
};

static TcShape tc_shape(int p)
{
    const int PP = p * p;
    if (PP <= 16) return {16, 1};
    if (PP <= 32) return {32, 1};
    if (PP <= 48) return {48, 2};
    if (PP <= 64) return {64, 2};
    if (PP <= 96) return {96, 3};
    if (PP <= 112) return {112, 4};
    if (PP <= 128) return {128, 4};
    return {0, 0};
}

bool tensor_m2l_supported(fmm_ctx *h) { return h->p >= 2 && tc_shape(h->p).NP > 0 && h->cc_major == 10; }

void tensor_tables_init(fmm_ctx *) {}

// T_v for every stencil vector: the real p^2 x p^2 map of M2L in the packed
// layout, L~_n^m = (-1)^n sum_{j,k} M~_j^k I_{j+n}^{k+m}(u), u = -v; split into
// TF32 (hi, lo) and laid out as the 128B-swizzled shared-memory image of the
// B operand: per k-block, rows 0..NP-1 = T_hi, rows NP..2NP-1 = T_lo.
static float tf32_rn_host(float a)
{
    uint32_t u;
    memcpy(&u, &a, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

// I_n^m(x) in full storage (n*n + n + m), degrees < Q, from the Cartesian
// recurrences of the irregular solid harmonics
static void build_irregular_full(int Q, double x, double y, double z, std::vector<double> &re, std::vector<double> &im)
{
    re.assign((size_t)Q * Q, 0.0);
    im.assign((size_t)Q * Q, 0.0);
    const double r2 = x * x + y * y + z * z, ir2 = 1.0 / r2;
    auto put = [&](int n, int m, double a, double b) {
        re[n * n + n + m] = a;
        im[n * n + n + m] = b;
        if (m) {
            const double sg = (m & 1) ? -1.0 : 1.0;
            re[n * n + n - m] = sg * a;
            im[n * n + n - m] = -sg * b;
        }
    };
    double mr = std::sqrt(ir2), mi = 0.0;
    for (int m = 0; m < Q; m++) {
        if (m > 0) {
            const double f = (double)(2 * m - 1) * ir2;
            const double a = (mr * x - mi * y) * f, b = (mr * y + mi * x) * f;
            mr = a;
            mi = b;
        }
        put(m, m, mr, mi);
        if (m + 1 >= Q) continue;
        const double f1 = (double)(2 * m + 1) * z * ir2;
        double p2r = mr, p2i = mi, p1r = mr * f1, p1i = mi * f1;
        put(m + 1, m, p1r, p1i);
        for (int n = m + 2; n < Q; n++) {
            const double a = (double)(2 * n - 1) * z, b = (double)((n + m - 1) * (n - m - 1));
            const double cr = (a * p1r - b * p2r) * ir2, ci = (a * p1i - b * p2i) * ir2;
            put(n, m, cr, ci);
            p2r = p1r;
            p2i = p1i;
            p1r = cr;
            p1i = ci;
        }
    }
}

void tensor_tables_update(fmm_ctx *h)
{
    const TcShape sh = tc_shape(h->p);
    if (!sh.NP) return;
    if (h->ttab_nv == h->nV && h->ttab.p) return;
    const int p = h->p, PP = p * p, Q = 2 * p - 1, NP = sh.NP, KB = sh.KB;
    const size_t bbytes = (size_t)2 * NP * 128;
    const size_t per_v = (size_t)KB * bbytes;
    std::vector<unsigned char> img((size_t)h->nV * per_v, 0);
    std::vector<int> seen(h->nV, 0);
    std::vector<double> Ire, Iim, T((size_t)PP * PP);
    auto re_i = [](int n, int m) { return n * n + (m == 0 ? 0 : 2 * m - 1); };
    auto im_i = [](int n, int m) { return n * n + 2 * m; };
    const int ne = h->st_off[8];
    for (int e = 0; e < ne; e++) {
        const int vx = h->st_host[4 * e], vy = h->st_host[4 * e + 1], vz = h->st_host[4 * e + 2], id = h->st_host[4 * e + 3];
        if (seen[id]) continue;
        seen[id] = 1;
        build_irregular_full(Q, -(double)vx, -(double)vy, -(double)vz, Ire, Iim);
        auto I = [&](int n, int m, double &r, double &i) {
            r = Ire[n * n + n + m];
            i = Iim[n * n + n + m];
        };
        std::fill(T.begin(), T.end(), 0.0);
        for (int j = 0; j < p; j++)
            for (int k = 0; k <= j; k++)
                for (int part = 0; part < (k ? 2 : 1); part++) {
                    // M_j^k = e (1 or i), M_j^{-k} = (-1)^k conj(e)
                    const double er = part ? 0.0 : 1.0, ei = part ? 1.0 : 0.0;
                    const int col = part ? im_i(j, k) : re_i(j, k);
                    for (int n = 0; n < p; n++)
                        for (int m = 0; m <= n; m++) {
                            double ir, ii, sr, si;
                            I(j + n, k + m, ir, ii);
                            sr = er * ir - ei * ii;
                            si = er * ii + ei * ir;
                            if (k) {
                                const double sg = (k & 1) ? -1.0 : 1.0;
                                double jr, ji;
                                I(j + n, m - k, jr, ji);
                                const double cr = sg * er, ci = -sg * ei;  // (-1)^k conj(e)
                                sr += cr * jr - ci * ji;
                                si += cr * ji + ci * jr;
                            }
                            if (n & 1) {
                                sr = -sr;
                                si = -si;
                            }
                            T[(size_t)re_i(n, m) * PP + col] = sr;
                            if (m) T[(size_t)im_i(n, m) * PP + col] = si;
                        }
                }
        unsigned char *dst = img.data() + (size_t)id * per_v;
        for (int r = 0; r < PP; r++)
            for (int c = 0; c < PP; c++) {
                const double t = T[(size_t)r * PP + c];
                const float hi = tf32_rn_host((float)t);
                const float lo = tf32_rn_host((float)(t - (double)hi));
                const int kb = c >> 5, cc = c & 31;
                for (int part = 0; part < 2; part++) {
                    const int row = r + part * NP;
                    const size_t off = (size_t)kb * bbytes + (size_t)row * 128 + (size_t)((((cc >> 2) ^ (row & 7)) << 4) + (cc & 3) * 4);
                    const float v = part ? lo : hi;
                    memcpy(dst + off, &v, 4);
                }
            }
    }
    h->ttab.ensure(img.size());
    FMM_CUDA_TRY(cudaMemcpy(h->ttab.p, img.data(), img.size(), cudaMemcpyHostToDevice));
    h->ttab_stride = per_v;
    h->ttab_nv = h->nV;
}

template <int NP, int KB>
static void launch_tc(fmm_ctx *h, float *L, const float *M)
{
    using C = TcCfg<NP, KB>;
    cudaStream_t s = h->work;
    const int c0 = h->depth >= 2 ? h->lvl_start[2] : h->ncells;
    const int nc = h->ncells;
    h->msplit.ensure(sizeof(float) * (size_t)nc * KB * 64);
    msplit_k<<<nblk((int64_t)(nc - c0) * KB * 32, 256), 256, 0, s>>>(M, h->p * h->p, KB, c0, nc, h->msplit.as<float>());
    count_launch(h);
    // stencil in shared memory when the largest octant stencil fits
    int nvmax = 0;
    for (int o = 0; o < 8; o++) nvmax = std::max(nvmax, h->st_off[o + 1] - h->st_off[o]);
    const int smem = 1024 + C::FIXED + (nvmax <= C::ST_MAX ? 16 * nvmax : 0);
    static int attr = 0;
    if (smem > attr) {
        FMM_CUDA_TRY(cudaFuncSetAttribute(m2l_tc_k<NP, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = smem;
    }
    const int *st_off = reinterpret_cast<const int *>(h->st_dev.as<char>() + sizeof(int4) * h->st_off[8]);
    const int *ntiles = reinterpret_cast<const int *>(h->m2l_misc.as<unsigned>() + 24 * (FMM_MAXLEVEL + 1));
    int *err = reinterpret_cast<int *>(h->m2l_misc.as<unsigned>() + 24 * (FMM_MAXLEVEL + 1) + 4);
    FMM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    m2l_tc_k<NP, KB><<<h->ntiles_max, 128, smem, s>>>(h->p, h->m2l_tiles.as<M2LTile>(), ntiles, h->m2l_tgt.as<int>(),
                                                         h->c_xyz.as<int4>(), h->c_anchor.as<uint64_t>(),
                                                         h->lvl_desc.as<LevelDesc>(), h->map_pool.as<int>(),
                                                         h->st_dev.as<int4>(), st_off, h->msplit.as<float>(),
                                                         h->ttab.as<unsigned char>(), L, err);
    count_launch(h);
    check_launch("m2l tensor");
}

void m2l_tensor(fmm_ctx *h, float *L, const float *M)
{
    tensor_tables_update(h);
    switch (tc_shape(h->p).NP) {
    case 16: launch_tc<16, 1>(h, L, M); break;
    case 32: launch_tc<32, 1>(h, L, M); break;
    case 48: launch_tc<48, 2>(h, L, M); break;
    case 64: launch_tc<64, 2>(h, L, M); break;
    case 96: launch_tc<96, 3>(h, L, M); break;
    case 112: launch_tc<112, 4>(h, L, M); break;
    case 128: launch_tc<128, 4>(h, L, M); break;
    default: throw Error{FMM_EINVAL, "tensor-core M2L: unsupported p"};
    }
}

}  // namespace fmm
