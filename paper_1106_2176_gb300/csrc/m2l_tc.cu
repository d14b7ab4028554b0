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
// Per CTA (320 threads: two groups of 4 worker warps, 1 MMA warp, 1 operator
// warp), for every unit (v, k-block) of 32 coefficients, taken by the group
// u % 2:
//   - the group gathers the unit's raw FP32 multipole rows with cp.async into
//     a 128B-swizzled stage of its A ring; each warp fills its own 32 rows,
//     eight lanes per row, so that one copy instruction covers four whole
//     rows (sources found by lattice lookups fetched ahead into a ring; zero
//     fill where a cell is absent);
//   - once the stage is full, each thread splits its row into TF32 hi and lo
//     (lo = a - hi), stores both in the unit's compute stage in tensor memory
//     and issues the copies of its group's next unit;
//   - the operator warp bulk-copies the pre-split, pre-swizzled [T_hi ; T_lo]
//     operator: for p <= 8 the blocks of a whole vector into a ring of its
//     own, several vectors ahead; otherwise one block into the unit's
//     compute stage;
//   - the MMA warp issues the tcgen05.mma (A from tensor memory, the operator
//     from shared memory) and commits; for p <= 8 it takes one whole vector
//     per iteration, waiting once on a barrier that both worker groups and the
//     operator warp arrive on, because every wait and commit costs the issuing
//     thread a few hundred cycles.
// Every wait is bounded; on a timeout the kernel records an error code and
// leaves after its copies have landed and its TMEM is released.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include <cuda.h>  // CUtensorMap and its encoding enums (the encoder comes from the runtime's driver entry point)

#include "fmm_internal.cuh"
#include "ptx_sm100.cuh"

namespace fmm {

static inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// source index of an absent cell, copied like a lattice-map entry
__device__ int g_no_cell = -1;

// ---------------------------------------------------------------------------
// tile geometry
// ---------------------------------------------------------------------------
// Warp roles: warps 0-7 form two groups of four (group g = warps 4g .. 4g+3,
// thread row r = tid % 128, in its warp's TMEM lane quarter); group g takes
// the units u with u % 2 == g, so the latency of one group's hand-offs is
// hidden behind the other's. Warp 8 issues the MMAs; warp 9 copies the
// operator blocks.
//   A raw rings (RSG stages per group, shared memory): the gathered FP32
//     multipoles of a unit, 128 B per row, 128B-swizzled. A warp copies and
//     reads only its own 32 rows, so it refills a stage right after the
//     warp's split.
//   compute stages (CS): A_hi, A_lo in tensor memory (written by the unit's
//     group with tcgen05.st, read by the MMA as its A operand), freed by the
//     MMA commit of the unit (or of its vector).
//   operator blocks in shared memory: VEC (p <= 8) a ring of OSV whole
//     vectors; otherwise one block in each compute stage.
// Tensor memory: AC accumulator buffers of 2 NP columns (main | correction)
// followed by the CS A stages of 64 columns (hi 32 | lo 32). Thread (r, g)
// drains output columns [g HN, (g + 1) HN) of row r.
template <int NP, int KB>
struct TcCfg {
    static constexpr int M = 128;                  // target rows per tile
    static constexpr int NW = 8;                   // worker warps
    static constexpr int NG = 2;                   // worker groups
    static constexpr int MMA_WARP = NW, B_WARP = NW + 1;
    static constexpr int NT = NW * 32 + 64;        // threads (workers, MMA warp, operator warp)
    static constexpr int A_RAW = M * 128;          // raw A k-block (FP32, swizzled)
    static constexpr int B_RAW = 2 * NP * 128;     // [T_hi ; T_lo] k-block (TF32 pair, swizzled)
    static constexpr int ACOLS = 64;               // TMEM columns of one A stage (hi, lo)
    // accumulator buffers: two (the drain overlaps the next MMAs) when the
    // compute stages of at least one whole vector (KB) still fit beside them
    static constexpr int CS2 = (512 - 4 * NP) / ACOLS >= 4 ? 4 : (512 - 4 * NP) / ACOLS;
    static constexpr int AC = CS2 >= KB && CS2 >= 2 ? 2 : 1;
    static constexpr int CS = AC == 2 ? CS2 : ((512 - 2 * NP) / ACOLS >= 4 ? 4 : (512 - 2 * NP) / ACOLS);
    static constexpr int ACC_COLS = AC * 2 * NP;
    static constexpr int TCOLS = 512;
    static constexpr int QU = 8;                   // lookahead of the source lookups (units of the group)
    static constexpr int RINGU = 2 * QU;
    static constexpr int RING = NG * RINGU * M * 4;
    // VEC (p <= 8): the MMA warp takes one stencil vector (KB units) per
    // iteration, and the operator blocks of whole vectors sit in a ring of
    // their own (OSV slots), filled up to OSV vectors ahead and freed by one
    // commit per vector (VR "vector done" barriers). Otherwise the operator
    // block of a unit travels in that unit's compute stage.
    static constexpr bool VEC = KB <= 2 && CS >= 2 * KB;
    static constexpr int OPV = KB * B_RAW;         // operator bytes of one vector
    static constexpr int VR = 8;
    static constexpr int RSG_V = 2;
    static constexpr int BAR = 768;                // mbarriers (first 512 bytes), then the CTA's job
    static constexpr int OSV_FIT = (220 * 1024 - RING - BAR - 1024 - NG * RSG_V * A_RAW) / OPV;
    static constexpr int OSV = OSV_FIT > 6 ? 6 : OSV_FIT;
    static constexpr int BUDGET = 220 * 1024 - RING - BAR - 1024 - CS * B_RAW;
    static constexpr int RSG_U = BUDGET / (NG * A_RAW) >= 3 ? 3 : BUDGET / (NG * A_RAW);
    static constexpr int RSG = VEC ? RSG_V : RSG_U;  // raw stages per group
    static constexpr int OPB = VEC ? OSV * OPV : CS * B_RAW;  // operator bytes in shared memory
    static constexpr int SMEM = NG * RSG * A_RAW + OPB + RING + BAR + 1024;
    static_assert(!VEC || (OSV >= 2 && OSV <= VR), "operator ring");
    static_assert(RSG >= 2 && RSG <= 3 && CS >= 2 && CS >= KB && QU >= RSG && ACC_COLS + CS * ACOLS <= TCOLS &&
                      SMEM <= 227 * 1024,
                  "stage budget");
    static constexpr int GV = 8;                   // vectors per accumulator drain
    static constexpr int HN = NP / 2;              // output coefficients per thread
    static constexpr int DRAIN_AT = AC == 2 ? 2 : 0;  // vectors into group gg + 1 at which group gg is drained
};

// Zero-padded copy of the scaled multipoles: out[c][KB * 32] (only when p^2 is
// not a multiple of 32; otherwise the kernel reads M~ directly).
__global__ void mpad_k(const float *__restrict__ M, int PP, int KP, int c0, int nc, float *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)(nc - c0) * KP) return;
    const int c = c0 + (int)(i / KP), k = (int)(i % KP);
    out[(size_t)c * KP + k] = k < PP ? M[(size_t)c * PP + k] : 0.f;
}

// Lattice copy of a complete level's M~ for the TMA tile loads of the
// tensor-core M2L: the row of the cell at lattice position (x, y, z) goes to
// ((b H + z/2) H + y/2) H + x/2, b = (x & 1) | (y & 1) << 1 | (z & 1) << 2 its
// octant bits and H = 2^(l-1), zero-padded to KP coefficients. The cells of
// one octant then form an H^3 block in x, y, z order, so the sources of a
// block of targets under one translation are a shifted block.
__global__ void lattice_fill_k(const float *__restrict__ M, int PP, int KP, const int4 *__restrict__ xyz, int c0, int c1,
                               int l, float *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)(c1 - c0) * KP) return;
    const int c = c0 + (int)(i / KP), k = (int)(i % KP);
    const int4 a = xyz[c];
    const int sh = FMM_MAXLEVEL - l;
    const int64_t H = 1ll << (l - 1);
    const int x = a.x >> sh, y = a.y >> sh, z = a.z >> sh;
    const int b = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
    const int64_t r = ((b * H + (z >> 1)) * H + (y >> 1)) * H + (x >> 1);
    out[r * KP + k] = k < PP ? M[(size_t)c * PP + k] : 0.f;
}

template <int NP, int KB, bool PERSIST>
__global__ void __launch_bounds__(TcCfg<NP, KB>::NT, 1)
    m2l_tc_k(int p, const __grid_constant__ M2LJob one, const M2LJob *__restrict__ jobs, int njobs,
             int *__restrict__ queue, int *__restrict__ err)
{
    // PERSIST (many systems: jobs[], njobs entries sorted by item0): each CTA
    // takes tiles from the queue until it is empty. Otherwise CTA b computes
    // tile b of the single job `one`, read from the parameter space, which
    // measured faster for one system than the persistent loop (25.1 vs
    // 27.7 ms at N = 1e7).
    using C = TcCfg<NP, KB>;
    constexpr int RSG = C::RSG, CS = C::CS, AC = C::AC, NG = C::NG, QU = C::QU, RINGU = C::RINGU, KP = KB * 32;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *araw = base;                           // NG x RSG x A_RAW
    constexpr bool VEC = C::VEC;
    constexpr int NB = VEC ? C::OSV : CS;     // operator slots
    constexpr int NF = VEC ? C::VR : CS;      // "free" barriers: per vector (VEC) or per compute stage
    unsigned char *bops = araw + NG * RSG * C::A_RAW;     // operator slots (VEC: OSV x OPV; else CS x B_RAW)
    int *ring = reinterpret_cast<int *>(bops + C::OPB);  // NG x RINGU x M
    uint64_t *bar = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(ring) + C::RING);
    uint64_t *a_full = bar;                   // NG x RSG: cp.async arrivals of the group's 128 threads
    uint64_t *b_full = a_full + NG * RSG;     // NB: operator copies (transaction bytes)
    uint64_t *cmp_full = b_full + NB;         // CS: one arrival per warp of the unit's group
    uint64_t *cmp_free = cmp_full + CS;       // NF: MMA commits (VEC: vector w done, slot w % VR)
    uint64_t *acc_full = cmp_free + NF;       // AC: MMA commits at the end of a group of vectors
    uint64_t *acc_empty = acc_full + AC;      // AC: one arrival per worker warp after a drain
    uint64_t *fin = acc_empty + AC;           // 1
    uint64_t *ready = fin + 1;                // VEC, VR: vector w ready (its KB units split, its operator landed)
    uint64_t *a_lat = ready + C::VR;          // NG x RSG x 4: TMA tile loads of one warp's 32 rows (lattice tiles)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(a_lat + NG * RSG * 4);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);
    int *s_tile = abort_flag + 1;                 // this CTA's current tile (-1: none left)
    M2LJob *s_job = reinterpret_cast<M2LJob *>(reinterpret_cast<unsigned char *>(bar) + 512);  // its job
    static_assert(sizeof(uint64_t) * (NG * RSG + NB + CS + NF + 2 * AC + 1 + C::VR + NG * RSG * 4) + 16 <= 512 &&
                      512 + sizeof(M2LJob) <= C::BAR,
                  "barrier area");

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool worker = warp < C::NW;
    const int row = tid & 127, grp = (tid >> 7) & 1;  // worker: target row and group
    if (warp == C::MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    for (int pass = 0; PERSIST || pass == 0; pass++) {
    if (tid == 0) {
        if (PERSIST) {
            const int it = atomicAdd(queue, 1);
            int lo = 0, hi = njobs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (jobs[mid].item0 <= it) lo = mid;
                else hi = mid - 1;
            }
            *s_job = jobs[lo];
            const int t = it - s_job->item0;
            *s_tile = (t >= 0 && t < s_job->count) ? t : -1;
        } else {
            *s_tile = (int)blockIdx.x < *one.ntiles ? (int)blockIdx.x : -1;
        }
        // the tile's barriers start from phase 0 (the previous tile left
        // every barrier idle: all its waits, copies and commits completed)
        for (int s = 0; s < NG * RSG; s++) mbar_init(&a_full[s], 128);
        for (int s = 0; s < NB; s++) mbar_init(&b_full[s], 1);
        for (int s = 0; s < CS; s++) mbar_init(&cmp_full[s], C::NW / C::NG);
        for (int s = 0; s < NF; s++) mbar_init(&cmp_free[s], 1);
        for (int b = 0; b < AC; b++) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], C::NW);
        }
        mbar_init(fin, 1);
        // per vector: one arrival per warp of the groups that split its KB
        // units, and one from the operator warp once the operator landed
        for (int s = 0; s < C::VR; s++) mbar_init(&ready[s], 4 * KB + 1);
        for (int s = 0; s < NG * RSG * 4; s++) mbar_init(&a_lat[s], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int tile = *s_tile;
    if (tile < 0) break;
    const M2LJob &J = PERSIST ? *s_job : one;
    const M2LTile *__restrict__ tiles = J.tiles;
    const int *__restrict__ tgt = J.tgt;
    const int4 *__restrict__ xyz = J.xyz;
    const uint64_t *__restrict__ anchor = J.anchor;
    const LevelDesc *__restrict__ ld = J.ld;
    const int *__restrict__ map_pool = J.map_pool;
    const int4 *__restrict__ st = J.st;
    const int *__restrict__ st_off = J.st_off;
    const float *__restrict__ mrow = J.mrow;
    const unsigned char *__restrict__ ttab = J.ttab;
    float *__restrict__ L = J.L;
    const M2LTile td = tiles[tile];
    const int PP = p * p;
    const int l = td.level;
    // this row's cell, its level, lattice position and octant (a pooled tile
    // mixes levels and octants)
    int px = 0, py = 0, pz = 0, cell = -1, rl = l, ro = 0;
    if (worker && row < td.count) {
        cell = tgt[td.start + row];
        const int4 a = xyz[cell];
        rl = a.w;
        const int sh = FMM_MAXLEVEL - rl;
        px = a.x >> sh;
        py = a.y >> sh;
        pz = a.z >> sh;
        ro = (px & 1) | ((py & 1) << 1) | ((pz & 1) << 2);
    }
    const LevelDesc LD = ld[rl];
    // the set's entries are sorted by reach: only a prefix can hit a cell
    const int e0 = st_off[td.octant], nv = st_off[10 + td.octant * (FMM_MAXLEVEL + 1) + l];
    const int nunits = nv * KB;
    const int ngroups = (nv + C::GV - 1) / C::GV;

    if (warp == C::MMA_WARP) {
        // ------------------------------------------------------------ MMA warp
        // VEC: one iteration per stencil vector (its KB compute stages and its
        // operator slot), so the waits and commits, a few hundred cycles each
        // on the issuing thread, are paid once per vector. Otherwise one
        // iteration per unit. The whole warp runs the loop; lane 0 issues.
        const uint32_t id_full = idesc_tf32(128, 2 * NP), id_half = idesc_tf32(128, NP);
        constexpr int STEP = VEC ? KB : 1;
        for (int u0 = 0; u0 < nunits; u0 += STEP) {
            const int vi = u0 / KB, g = vi / C::GV, b = g % AC;
            bool ok = true;
#pragma unroll
            for (int kb = 0; kb < (VEC ? 0 : STEP); kb++) ok = ok && mbar_wait(&cmp_full[(u0 + kb) % CS], (uint32_t)(((u0 + kb) / CS) & 1));
            if (VEC) ok = mbar_wait(&ready[vi % C::VR], (uint32_t)((vi / C::VR) & 1));
            if (ok && u0 % KB == 0 && vi % C::GV == 0 && g >= AC) ok = mbar_wait(&acc_empty[b], (uint32_t)(((g - AC) / AC) & 1));
            ok = __all_sync(0xffffffffu, ok) && !*(volatile int *)abort_flag;
            if (!ok) {
                if (lane == 0) atomicExch(abort_flag, 1);
                break;
            }
            tc_fence_after();
            if (lane == 0) {
                const uint32_t dmain = tmem + (uint32_t)(b * 2 * NP), dcorr = dmain + NP;
                const bool first = vi % C::GV == 0;
#pragma unroll
                for (int kk = 0; kk < STEP; kk++) {
                    const int u = u0 + kk, c = u % CS, kb = u % KB;
                    const uint32_t ahi = tmem + (uint32_t)(C::ACC_COLS + c * C::ACOLS), alo = ahi + 32;
                    const uint32_t bb = VEC ? smem_u32(bops + (vi % NB) * C::OPV + kb * C::B_RAW) : smem_u32(bops + c * C::B_RAW);
                    // k-steps of 8 coefficients holding any of the p^2 real ones: the
                    // rest of a padded k-block is zero in A and in the operator and
                    // would add exactly zero (p = 6: 5 of 8 k-steps; p = 8: all)
                    const int ks = min(4, (PP - kb * 32 + 7) >> 3);
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        if (k >= ks) break;
                        // A_hi [T_hi ; T_lo] -> main | correction, then A_lo T_hi -> correction
                        mma_tf32_ta(dmain, ahi + 8 * k, sdesc(bb + 32 * k), id_full, (first && kb == 0 && k == 0) ? 0u : 1u);
                        mma_tf32_ta(dcorr, alo + 8 * k, sdesc(bb + 32 * k), id_half, 1u);
                    }
                }
                if (VEC) mma_commit(&cmp_free[vi % NF]);
                else mma_commit(&cmp_free[u0 % CS]);
                if ((u0 + STEP) % KB == 0 && ((vi % C::GV == C::GV - 1) || vi == nv - 1)) mma_commit(&acc_full[b]);
            }
            __syncwarp();
        }
        if (lane == 0) {
            // every commit has arrived before the shared memory goes away
            mma_commit(fin);
            mbar_wait(fin, 0);
            if (VEC)
                for (int w = max(0, nv - NF); w < nv; w++) mbar_wait(&cmp_free[w % NF], (uint32_t)((w / NF) & 1));
            else
                for (int u = max(0, nunits - CS); u < nunits; u++) mbar_wait(&cmp_free[u % CS], (uint32_t)((u / CS) & 1));
        }
        __syncwarp();
    } else if (warp == C::B_WARP) {
        // ------------------------------------------------------- operator warp
        // VEC: the vector's KB operator blocks (contiguous in the image) in one
        // bulk copy into slot w % OSV, once vector w - OSV is done. Otherwise
        // one block per unit into its compute stage, once that stage is free.
        if (lane == 0) {
            int issued = 0;
            const int nitems = VEC ? nv : nunits;
            for (int w = 0; w < nitems; w++) {
                if (*(volatile int *)abort_flag) break;
                bool ok = true;
                if (VEC) {
                    if (w >= NB) ok = mbar_wait(&cmp_free[(w - NB) % NF], (uint32_t)(((w - NB) / NF) & 1));
                } else if (w >= CS) {
                    ok = mbar_wait(&cmp_free[w % CS], (uint32_t)(((w - CS) / CS) & 1));
                }
                if (!ok) {
                    atomicExch(abort_flag, 1);
                    break;
                }
                const int bs = w % NB;
                if (VEC) {
                    const int4 v = st[e0 + w];
                    mbar_arrive_tx(&b_full[bs], C::OPV);
                    bulk_g2s(smem_u32(bops + bs * C::OPV), ttab + (size_t)(v.w & 0xffff) * C::OPV, C::OPV, &b_full[bs]);
                    // vector w - 1's operator has landed: its readiness
                    if (w >= 1) {
                        if (!mbar_wait(&b_full[(w - 1) % NB], (uint32_t)(((w - 1) / NB) & 1))) {
                            atomicExch(abort_flag, 1);
                            issued = w + 1;
                            break;
                        }
                        mbar_arrive(&ready[(w - 1) % C::VR]);
                    }
                } else {
                    const int4 v = st[e0 + w / KB];
                    mbar_arrive_tx(&b_full[bs], C::B_RAW);
                    bulk_g2s(smem_u32(bops + bs * C::B_RAW), ttab + ((size_t)(v.w & 0xffff) * KB + w % KB) * C::B_RAW,
                             C::B_RAW, &b_full[bs]);
                }
                issued = w + 1;
            }
            if (VEC && issued == nitems && nitems > 0 && !*(volatile int *)abort_flag) {
                if (mbar_wait(&b_full[(nitems - 1) % NB], (uint32_t)(((nitems - 1) / NB) & 1)))
                    mbar_arrive(&ready[(nitems - 1) % C::VR]);
                else
                    atomicExch(abort_flag, 1);
            }
            // copies still in flight when the pipeline stopped early land
            // before the shared memory goes away (bounded waits)
            if (*(volatile int *)abort_flag)
                for (int w = max(0, issued - NB); w < issued; w++) mbar_wait(&b_full[w % NB], (uint32_t)((w / NB) & 1));
        }
    } else {
        // ---------------------------------------------------------- worker warps
        constexpr int HN = C::HN;
        float acc_hi[HN], acc_lo[HN];
#pragma unroll
        for (int k = 0; k < HN; k++) acc_hi[k] = acc_lo[k] = 0.f;
        const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;  // this warp's TMEM lane quarter
        const int g = grp;
        const int nown = nunits > g ? (nunits - g + 1) / 2 : 0;  // units u = g, g + 2, ... of this group
        int *myring = ring + g * RINGU * C::M;
        const bool dense = LD.map_off >= 0;  // the level has a lattice map: lookups arrive by cp.async
        const bool full = rl <= 10 && LD.end - LD.start == (1 << (3 * rl));  // every lattice cell present
        // Lattice tile (a complete level with a lattice copy of M~): the tile
        // is an 8 x 4 x 4 block of its octant's sub-lattice with rows in x, y,
        // z order, and for every vector the sources form the same block
        // shifted, in the sub-lattice of the source octant. Each warp brings
        // its 32 rows (one z slice) with one TMA tile load; positions outside
        // the level arrive as zeros, like absent cells.
        // (persistent launches serve the batch engine, which gathers everywhere)
        const bool lat = !PERSIST && J.lat_maps != nullptr && td.octant < 8 && ((J.lat_levels >> l) & 1u);
        const int q = warp & 3;
        const int obx = td.octant & 1, oby = (td.octant >> 1) & 1, obz = (td.octant >> 2) & 1;
        // tile origin in halved coordinates (from row 32 q = (0, 0, q), this warp's lane 0)
        const int ox = (px >> 1) - (row & 7), oy = (py >> 1) - ((row >> 3) & 3), oz = (pz >> 1) - (row >> 5);
        const void *lmap = lat ? (const void *)(J.lat_maps + 128 * l) : nullptr;
        int lat_issued = 0, lat_done = 0;  // this warp's TMA loads issued / waited for

        // source cell of this row for the group's unit j, looked up QU units
        // ahead into ring slot j % RINGU (cp.async of the lattice-map entry, or
        // a search of the level's keys); only this thread reads the slot, after
        // the raw-stage barrier that its own later copies arrive on
        // stencil entry of the group's unit j; the next call's entry is
        // loaded one call ahead (calls come in order), so its latency is hidden
        int4 st_next = make_int4(0, 0, 0, 0);
        int st_next_j = -1;
        auto fetch = [&](int j) {
            if (lat || j >= nown) return;
            const int4 v = st_next_j == j ? st_next : st[e0 + (2 * j + g) / KB];
            if (j + 1 < nown) {
                st_next = st[e0 + (2 * (j + 1) + g) / KB];
                st_next_j = j + 1;
            }
            const uint32_t slot = smem_u32(myring + (j % RINGU) * C::M + row);
            int r = -1;
            if (cell >= 0) {
                const int x = px + v.x, y = py + v.y, z = pz + v.z, side = 1 << rl;
                if (((v.w >> (16 + ro)) & 1) && x >= 0 && y >= 0 && z >= 0 && x < side && y < side && z < side) {
                    // a complete level holds every lattice cell in Morton order:
                    // the index follows from the position
                    if (full) {
                        myring[(j % RINGU) * C::M + row] = LD.start + (int)morton3_10((uint32_t)x, (uint32_t)y, (uint32_t)z);
                        return;
                    }
                    if (dense) {
                        cp_async4(slot, map_pool + LD.map_off + (long long)morton3((uint32_t)x, (uint32_t)y, (uint32_t)z));
                        return;
                    }
                    r = level_lookup(LD, map_pool, anchor, rl, x, y, z);
                }
            }
            if (dense && !full) cp_async4(slot, &g_no_cell);
            else myring[(j % RINGU) * C::M + row] = r;
        };
        // copy the group's unit j into its raw stage j % RSG. The warp fills
        // its own 32 rows: in copy i, lanes 8s .. 8s+7 take the eight 16-byte
        // chunks of row 4i + s, so one warp instruction reads 4 whole rows
        // (4 cache lines, not 32); the source of each row comes from the lane
        // that looked it up
        auto load_unit = [&](int j) {
            const int u = 2 * j + g, kb = u % KB;
            if (lat) {
                // the stencil entry of this call is loaded one call ahead (the
                // lookahead registers of the lookups, which lattice tiles skip)
                if (lane == 0) {
                    const int4 v = st_next_j == j ? st_next : st[e0 + u / KB];
                    if (j + 1 < nown) {
                        st_next = st[e0 + (u + 2) / KB];
                        st_next_j = j + 1;
                    }
                    // source octant bits and the block's shift in halved
                    // coordinates (arithmetic shifts: floor division by 2)
                    const int sx = obx + v.x, sy = oby + v.y, sz = obz + v.z;
                    const int ps = (sx & 1) | ((sy & 1) << 1) | ((sz & 1) << 2);
                    uint64_t *b = &a_lat[(g * RSG + j % RSG) * 4 + q];
                    // the warp's generic reads of this stage precede the async-proxy writes
                    fence_proxy_async();
                    mbar_arrive_tx(b, 32 * 128);
                    tma_load_5d(smem_u32(araw + (g * RSG + j % RSG) * C::A_RAW + q * 32 * 128), lmap, kb * 32,
                                ox + (sx >> 1), oy + (sy >> 1), oz + q + (sz >> 1), ps, b);
                }
                lat_issued = j + 1;
                return;
            }
            const int src = myring[(j % RINGU) * C::M + row];
            fetch(j + QU);
            const uint32_t ab = smem_u32(araw + (g * RSG + j % RSG) * C::A_RAW);
            const int ch = lane & 7, sub = lane >> 3, r0 = row - lane;  // r0: the warp's first row
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const int rr = r0 + 4 * i + sub;
                const int s = __shfl_sync(0xffffffffu, src, 4 * i + sub);
                const float *gs = mrow + ((size_t)(s >= 0 ? s : 0) * KP + kb * 32) + ch * 4;
                cp_async16(ab + (uint32_t)rr * 128u + ((((uint32_t)ch) ^ ((uint32_t)rr & 7u)) << 4), gs, s >= 0 ? 16u : 0u);
            }
            cp_async_arrive_noinc(&a_full[g * RSG + j % RSG]);
        };

        auto drain = [&](int gg) {
            const int b = gg % AC;
            __syncwarp();
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], (uint32_t)((gg / AC) & 1)));
            if (!ok) {
                atomicExch(abort_flag, 1);
                return;
            }
            tc_fence_after();
            const uint32_t taddr = tmem + tlane + (uint32_t)(b * 2 * NP + g * HN);
            float mv[16], cv[16];
#pragma unroll
            for (int k0 = 0; k0 < HN; k0 += 16) {
                if (k0 + 16 <= HN) {
                    tmem_ld16(taddr + k0, mv);
                    tmem_ld16(taddr + NP + k0, cv);
                } else {  // 8 remaining columns
                    tmem_ld8(taddr + k0, mv);
                    tmem_ld8(taddr + NP + k0, cv);
                }
#pragma unroll
                for (int k = 0; k < 16; k++)
                    if (k0 + k < HN) two_sum_acc(acc_hi[k0 + k], acc_lo[k0 + k], mv[k] + cv[k]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        };

        for (int j = 0; j < QU; j++) fetch(j);
        cp_async_commit();
        cp_async_wait_all();
        for (int j = 0; j < RSG && j < nown; j++) load_unit(j);
        int drained = 0;
        for (int j = 0; j < nown; j++) {
            if (*(volatile int *)abort_flag) break;
            const int u = 2 * j + g, c = u % CS, vi = u / KB;
            // one accumulator buffer: group gg is drained before group gg + 1 starts
            if (AC == 1 && vi / C::GV > drained) {
                drain(drained);
                drained++;
                if (*(volatile int *)abort_flag) break;
            }
            // the compute stage is free once the unit that used it last (u - CS)
            // is done: its vector's commit (VEC) or its own (otherwise)
            const int wprev = max(u - CS, 0) / KB;
            uint64_t *araw_bar = lat ? &a_lat[(g * RSG + j % RSG) * 4 + q] : &a_full[g * RSG + j % RSG];
            const bool ok = VEC ? mbar_wait2(u >= CS ? 3u : 1u, araw_bar, (uint32_t)((j / RSG) & 1),
                                             &cmp_free[wprev % NF], (uint32_t)((wprev / NF) & 1))
                                : mbar_wait2(u >= CS ? 3u : 1u, araw_bar, (uint32_t)((j / RSG) & 1),
                                             &cmp_free[c], (uint32_t)((max(u - CS, 0) / CS) & 1));
            if (!ok) {
                atomicExch(abort_flag, 1);
                break;
            }
            lat_done = j + 1;
            tc_fence_after();
            // split this row's raw FP32 k-block into TF32 (hi, lo): hi rounded to
            // nearest, lo = a - hi (exact in FP32; the MMA reads its leading 11
            // bits, an error below 2^-21 of a); both go to the A stage in TMEM
            const unsigned char *rs = araw + (g * RSG + j % RSG) * C::A_RAW + row * 128;
            const uint32_t ta = tmem + tlane + (uint32_t)(C::ACC_COLS + c * C::ACOLS);
            // the second half of a k-block that holds only padding is never read
            // by the MMAs (they skip its k-steps)
            const int nh = (u % KB) * 32 + 16 < PP ? 2 : 1;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                if (h >= nh) break;
                float hi[16], lo[16];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int ch = 4 * h + q;
                    const float4 a = *reinterpret_cast<const float4 *>(rs + ((ch ^ (row & 7)) << 4));
                    hi[4 * q + 0] = tf32_rn(a.x); lo[4 * q + 0] = a.x - hi[4 * q + 0];
                    hi[4 * q + 1] = tf32_rn(a.y); lo[4 * q + 1] = a.y - hi[4 * q + 1];
                    hi[4 * q + 2] = tf32_rn(a.z); lo[4 * q + 2] = a.z - hi[4 * q + 2];
                    hi[4 * q + 3] = tf32_rn(a.w); lo[4 * q + 3] = a.w - hi[4 * q + 3];
                }
                tmem_st16(ta + 16 * h, hi);
                tmem_st16(ta + 32 + 16 * h, lo);
            }
            // every lane of the warp has read its row of the raw stage: the
            // next unit's copies may overwrite it while the stores complete
            __syncwarp();
            if (j + RSG < nown) load_unit(j + RSG);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                // (per unit) the group's first warp also waits for the operator block
                if (!VEC && (warp & 3) == 0 && !mbar_wait(&b_full[c], (uint32_t)((u / CS) & 1))) atomicExch(abort_flag, 1);
                mbar_arrive(VEC ? &ready[(u / KB) % C::VR] : &cmp_full[c]);
            }
            // two accumulator buffers: drain group gg once group gg + 1 is well under way
            if (AC == 2 && vi >= C::DRAIN_AT && (vi - C::DRAIN_AT) / C::GV > drained) {
                drain(drained);
                drained++;
            }
        }
        cp_async_wait_all();
        // tile loads still in flight when the loop stopped early land before
        // the shared memory is reused or released (bounded waits)
        if (lat && lane == 0)
            for (int jj = lat_done; jj < lat_issued; jj++)
                mbar_wait(&a_lat[(g * RSG + jj % RSG) * 4 + q], (uint32_t)((jj / RSG) & 1));
        __syncwarp();
        if (!*(volatile int *)abort_flag) {
            while (drained < ngroups) {
                drain(drained);
                drained++;
                if (*(volatile int *)abort_flag) break;
            }
        }
        if (cell >= 0 && !*(volatile int *)abort_flag) {
            float *Lc = L + (size_t)cell * PP + g * HN;
#pragma unroll
            for (int k = 0; k < HN; k++)
                if (g * HN + k < PP) Lc[k] += acc_hi[k] + acc_lo[k];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const bool aborted = *(volatile int *)abort_flag != 0;
    if (tid == 0 && aborted) atomicExch(err, 1);
    __syncthreads();  // every thread has read the flag before the next tile resets it
    if (aborted) break;
    }  // tiles
    tc_fence_before();
    __syncthreads();
    if (warp == C::MMA_WARP) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TCOLS));
    }
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

// The operator image depends only on p and the stencil, which the MAC
// constant and the stencil bound fix (vectors are numbered in a fixed order):
// handles with the same three share one host image, built once per process.
static std::mutex g_img_mu;
static std::map<std::tuple<int, double, int>, std::shared_ptr<const std::vector<unsigned char>>> g_img_cache;

void tensor_tables_update(fmm_ctx *h)
{
    const TcShape sh = tc_shape(h->p);
    if (!sh.NP) return;
    if (h->ttab_nv == h->nV && h->ttab.p) return;
    const auto key = std::make_tuple(h->p, h->cmac, h->st_R);
    {
        std::lock_guard<std::mutex> lk(g_img_mu);
        auto it = g_img_cache.find(key);
        if (it != g_img_cache.end()) {
            h->ttab.ensure(it->second->size());
            FMM_CUDA_TRY(cudaMemcpy(h->ttab.p, it->second->data(), it->second->size(), cudaMemcpyHostToDevice));
            h->ttab_stride = (size_t)tc_shape(h->p).KB * 2 * tc_shape(h->p).NP * 128;
            h->ttab_nv = h->nV;
            return;
        }
    }
    const int p = h->p, PP = p * p, Q = 2 * p - 1, NP = sh.NP, KB = sh.KB;
    const size_t bbytes = (size_t)2 * NP * 128;  // one k-block of [T_hi ; T_lo]
    const size_t per_v = (size_t)KB * bbytes;
    std::vector<unsigned char> img((size_t)h->nV * per_v, 0);
    std::vector<int> seen(h->nV, 0);
    std::vector<double> Ire, Iim, T((size_t)PP * PP);
    auto re_i = [](int n, int m) { return n * n + (m == 0 ? 0 : 2 * m - 1); };
    auto im_i = [](int n, int m) { return n * n + 2 * m; };
    const int ne = h->st_off[8];
    for (int e = 0; e < ne; e++) {
        const int vx = h->st_host[4 * e], vy = h->st_host[4 * e + 1], vz = h->st_host[4 * e + 2], id = h->st_host[4 * e + 3] & 0xffff;
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
        // per k-block the 128B-swizzled image of [T_hi ; T_lo]: rows 0..NP-1
        // hold hi = TF32(T) (round to nearest), rows NP..2NP-1 lo = T - hi
        unsigned char *dst = img.data() + (size_t)id * per_v;
        for (int r = 0; r < PP; r++)
            for (int c = 0; c < PP; c++) {
                const double t = T[(size_t)r * PP + c];
                const float hi = tf32_rn_host((float)t);
                const float lo = (float)(t - (double)hi);
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
    std::lock_guard<std::mutex> lk(g_img_mu);
    g_img_cache[key] = std::make_shared<const std::vector<unsigned char>>(std::move(img));
}

template <int NP, int KB>
static void launch_tc(int p, int grid, const M2LJob &one, const M2LJob *jobs, int njobs, int *queue, int *err,
                      cudaStream_t s)
{
    using C = TcCfg<NP, KB>;
    // grid: one CTA per SM with a job list (persistent), else one per tile
    if (jobs) {
        ensure_smem((const void *)m2l_tc_k<NP, KB, true>, C::SMEM);
        FMM_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(int), s));
        m2l_tc_k<NP, KB, true><<<grid, C::NT, C::SMEM, s>>>(p, one, jobs, njobs, queue, err);
    } else {
        ensure_smem((const void *)m2l_tc_k<NP, KB, false>, C::SMEM);
        m2l_tc_k<NP, KB, false><<<grid, C::NT, C::SMEM, s>>>(p, one, jobs, njobs, queue, err);
    }
}

static void launch_tc_p(int p, int nsm, const M2LJob &one, const M2LJob *jobs, int njobs, int *queue, int *err,
                        cudaStream_t s)
{
    switch (tc_shape(p).NP) {
    case 16: launch_tc<16, 1>(p, nsm, one, jobs, njobs, queue, err, s); break;
    case 32: launch_tc<32, 1>(p, nsm, one, jobs, njobs, queue, err, s); break;
    case 48: launch_tc<48, 2>(p, nsm, one, jobs, njobs, queue, err, s); break;
    case 64: launch_tc<64, 2>(p, nsm, one, jobs, njobs, queue, err, s); break;
    case 96: launch_tc<96, 3>(p, nsm, one, jobs, njobs, queue, err, s); break;
    case 112: launch_tc<112, 4>(p, nsm, one, jobs, njobs, queue, err, s); break;
    case 128: launch_tc<128, 4>(p, nsm, one, jobs, njobs, queue, err, s); break;
    default: throw Error{FMM_EINVAL, "tensor-core M2L: unsupported p"};
    }
}

M2LJob m2l_tensor_job(fmm_ctx *h, float *L, const float *M, cudaStream_t s)
{
    tensor_tables_update(h);
    const TcShape sh = tc_shape(h->p);
    const int c0 = h->depth >= 2 ? h->lvl_start[2] : h->ncells;
    const int nc = h->ncells, PP = h->p * h->p, KP = sh.KB * 32;
    const float *mrow = M;
    if (PP != KP) {  // zero-padded rows of KB * 32 coefficients
        h->msplit.ensure(sizeof(float) * (size_t)nc * KP);
        if (nc > c0) {
            mpad_k<<<nblk((int64_t)(nc - c0) * KP, 256), 256, 0, s>>>(M, PP, KP, c0, nc, h->msplit.as<float>());
            count_launch(h);
        }
        mrow = h->msplit.as<float>();
    }
    M2LJob j;
    j.tiles = h->m2l_tiles.as<M2LTile>();
    j.ntiles = reinterpret_cast<const int *>(h->m2l_misc.as<unsigned>() + 24 * (FMM_MAXLEVEL + 1));
    j.tgt = h->m2l_tgt.as<int>();
    j.xyz = h->c_xyz.as<int4>();
    j.anchor = h->c_anchor.as<uint64_t>();
    j.ld = h->lvl_desc.as<LevelDesc>();
    j.map_pool = h->map_pool.as<int>();
    j.st = h->st_dev.as<int4>();
    j.st_off = stencil_offsets(h);
    j.mrow = mrow;
    j.ttab = h->ttab.as<unsigned char>();
    j.L = L;
    j.lat_maps = nullptr;  // gathers on every level (the single-system launch sets the lattice levels)
    j.lat_levels = 0;
    j.item0 = 0;
    j.count = -1;
    return j;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link
// against the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

// The complete levels whose tiles are lattice blocks (at least 8^4 cells,
// more than the pooling threshold, so every tile is 128 cells of one octant)
// read their sources by TMA from a lattice copy of M~: one 5-D tensor map per
// level over [octant bits][z/2][y/2][x/2][KP coefficients] (FP32), box
// 32 coefficients x 8 x 4 x 1 x 1 = one warp's 32 rows, 128-byte swizzle
// (the layout of the gathered stages). Levels beyond 9 keep the gathers.
void lattice_prepare(fmm_ctx *h, cudaStream_t s)
{
    h->lat_levels = 0;
    if (!h->lattice_req || h->precision != FMM_MIXED || h->engine_used != FMM_M2L_TENSOR || !tensor_m2l_supported(h) ||
        m2l_tile_size(h) != TcCfg<64, 2>::M)
        return;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return;
    const int KP = tc_shape(h->p).KB * 32;
    const int pool_max = h->m2l_pool >= 0 ? h->m2l_pool : 4 * m2l_tile_size(h);
    unsigned levels = 0;
    long long total = 0;
    for (int l = 4; l <= std::min(h->depth, 9); l++) {
        const long long cells = (long long)h->lvl_start[(size_t)l + 1] - h->lvl_start[(size_t)l];
        if (cells != (1ll << (3 * l)) || cells <= pool_max) continue;
        levels |= 1u << l;
        h->lat_off[l] = total;
        total += cells * KP;
    }
    if (!levels) return;
    h->mlat.ensure(sizeof(float) * (size_t)total);
    const size_t mbytes = sizeof(CUtensorMap) * (FMM_MAXLEVEL + 1);
    h->lat_maps.ensure(mbytes);
    h->lat_host.ensure(mbytes);
    CUtensorMap *mp = h->lat_host.as<CUtensorMap>();
    std::memset(mp, 0, mbytes);
    for (int l = 4; l <= 9; l++) {
        if (!((levels >> l) & 1u)) continue;
        const cuuint64_t H = 1ull << (l - 1), row = sizeof(float) * (cuuint64_t)KP;
        const cuuint64_t dims[5] = {(cuuint64_t)KP, H, H, H, 8};
        const cuuint64_t strides[4] = {row, row * H, row * H * H, row * H * H * H};
        const cuuint32_t box[5] = {32, 8, 4, 1, 1}, estride[5] = {1, 1, 1, 1, 1};
        const CUresult r = enc(&mp[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, h->mlat.as<float>() + h->lat_off[l], dims,
                               strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) throw Error{FMM_ECUDA, "tensor-core M2L: encoding a lattice tensor map failed"};
    }
    FMM_CUDA_TRY(cudaMemcpyAsync(h->lat_maps.p, mp, mbytes, cudaMemcpyHostToDevice, s));
    h->lat_levels = levels;
}

__global__ void batch_mpad_k(int PP, int KP, const BatchSys *__restrict__ sys)
{
    const BatchSys &S = sys[blockIdx.y];
    if (!S.mpad || S.c0 >= S.ncells) return;
    const int64_t cnt = (int64_t)(S.ncells - S.c0) * KP;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = S.c0 + (int)(i / KP), k = (int)(i % KP);
        S.mpad[(size_t)c * KP + k] = k < PP ? S.M[(size_t)c * PP + k] : 0.f;
    }
}

void batch_mpad(int p, const BatchSys *sys, int nsys, cudaStream_t s)
{
    const int PP = p * p, KP = tc_shape(p).KB * 32;
    if (PP == KP) return;
    batch_mpad_k<<<dim3(16, (unsigned)nsys), 256, 0, s>>>(PP, KP, sys);
    check_launch("batch pad");
}

void m2l_tensor_jobs(int p, int nsm, const M2LJob *jobs_dev, int njobs, int *queue, int *err, cudaStream_t s)
{
    M2LJob none;
    std::memset(&none, 0, sizeof(none));
    launch_tc_p(p, nsm, none, jobs_dev, njobs, queue, err, s);
}

void m2l_tensor(fmm_ctx *h, float *L, const float *M)
{
    cudaStream_t s = h->work;
    M2LJob j = m2l_tensor_job(h, L, M, s);
    if (h->lat_levels) {
        const int PP = h->p * h->p, KP = tc_shape(h->p).KB * 32;
        for (int l = 0; l <= FMM_MAXLEVEL; l++) {
            if (!((h->lat_levels >> l) & 1u)) continue;
            const int c0 = h->lvl_start[(size_t)l], c1 = h->lvl_start[(size_t)l + 1];
            lattice_fill_k<<<nblk((int64_t)(c1 - c0) * KP, 256), 256, 0, s>>>(M, PP, KP, h->c_xyz.as<int4>(), c0, c1, l,
                                                                            h->mlat.as<float>() + h->lat_off[l]);
            count_launch(h);
        }
        j.lat_maps = h->lat_maps.as<unsigned char>();
        j.lat_levels = h->lat_levels;
    }
    int *misc = reinterpret_cast<int *>(h->m2l_misc.as<unsigned>() + 24 * (FMM_MAXLEVEL + 1));
    int *err = misc + 4, *queue = misc + 6;
    FMM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    launch_tc_p(h->p, h->ntiles_max, j, nullptr, 1, queue, err, s);
    count_launch(h);
    check_launch("m2l tensor");
}

}  // namespace fmm
