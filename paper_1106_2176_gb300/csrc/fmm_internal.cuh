// Internal declarations of the GB300 FMM library (not part of the C ABI).
//
// Data layout in HBM (one handle, n particles, C cells, p terms, PP = p*p):
//   sorted particles   xs64[n] double4_32a (x, y, z, q)      FP64 path, FP64 input
//                      xs32[n] float4  (x, y, z, q)      mixed path (P2P)
//                      xs32lo[n] float4 (x - fl(x), ...)  mixed path, FP64 input
//   cells (SoA, breadth first, key order within a level)
//                      level, begin, end, child, nchild, parent: int32[C]
//                      anchor: uint64[C] (Morton key of the lowest corner)
//                      xyz: int4[C] (lowest corner in grid units, level)
//   expansions         Mexp, Lexp: real[C][PP], packed real layout (degree n at
//                      offset n*n: Re(n,0), Re(n,1), Im(n,1), ..., Re(n,n), Im(n,n)),
//                      scaled by the cell width w: M_n^m / w^n, L_n^m w^(n+1)
//   lists              P2P: CSR by target cell, int32 sources ascending
//                      M2L between cells of different levels: CSR, int32
//                      M2L between cells of one level: implicit, the stencil
//                      of the target's octant applied through a per-level map
//   results            far[n], near[n]: double4_32a (phi, dphi/dx, dphi/dy, dphi/dz)
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/fmm.h"

#define FMM_MAXP 20
#define FMM_MAXLEVEL 21
#define FMM_DENSE_MAP_MAXLEVEL 8  // levels with 8^l <= 2^24 get a dense lattice map

namespace fmm {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
struct Error {
    int code;
    std::string msg;
};

void set_error(const std::string &msg);
const std::string &get_error();

#define FMM_CUDA_TRY(expr)                                                                 \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            throw ::fmm::Error{FMM_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

// ---------------------------------------------------------------------------
// device memory owned by a handle; grows on demand, never shrinks
// ---------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    void ensure(size_t bytes);  // may reallocate (contents are not kept)
    void ensure_keep(size_t bytes, size_t used, cudaStream_t s);  // keeps the first `used` bytes
    void release();
    template <class T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

struct PinnedBuf {
    void *p = nullptr;
    size_t cap = 0;
    void ensure(size_t bytes);
    void release();
    template <class T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

// root cube, computed on the device
struct Box {
    unsigned long long enc_lo[3], enc_hi[3];  // order-preserving encodings of min / max
    double origin[3];
    double R0;     // half width of the root cube
    double s;      // 2^21 / (2 R0)
    double h;      // 2 R0 / 2^21 (grid spacing)
    int nonfinite; // set when a coordinate is NaN or infinite
    int pad;
};

// open-addressed table slot: Morton index of a cell at its level plus one
// (0: empty), and the cell
struct HashSlot {
    unsigned long long key;
    int val, pad;
};

// per-level lookup from lattice position to cell index (M2L stencil)
struct LevelDesc {
    int start, end;         // cell index range of the level
    long long map_off;      // offset of a dense map (8^l int32) in the map pool, or -1
    const HashSlot *hash;   // levels without a dense map: a table of at least twice their cells, or null
    unsigned hash_mask;     // table size - 1 (a power of two)
    int pad;
};

// M2L tile: up to TILE target cells of one level and one octant, or (octant
// 8) cells of the sparse levels of every octant, level their largest level
struct M2LTile {
    int start;   // first entry in the target list
    int count;
    int level;
    int octant;
};

// One system's share of a persistent tensor-core M2L launch: its tile list
// and the arrays the tiles read and write. Queue items item0 .. item0 + count
// - 1 are its tiles (count < 0: *ntiles tiles, read on the device).
struct M2LJob {
    const M2LTile *tiles;
    const int *ntiles;
    const int *tgt;
    const int4 *xyz;
    const uint64_t *anchor;
    const LevelDesc *ld;
    const int *map_pool;
    const int4 *st;
    const int *st_off;
    const float *mrow;
    const unsigned char *ttab;
    float *L;
    // complete levels whose sources come by TMA tile loads from the lattice
    // copy of M~ (bit l: level l); lat_maps holds a 128-byte tensor map per level
    const unsigned char *lat_maps;
    unsigned lat_levels;
    int item0;
    int count;
};

// One system of a batched evaluation (mixed precision, FP32 inputs): the
// arrays of its handle that the batch kernels read and write, its output
// buffers and its dependency counters.
struct BatchSys {
    const int *leaves, *begin, *end, *child, *nchild, *parent, *pcell, *inv;
    const int4 *xyz;
    const Box *box;
    const double4_32a *cgeo;
    const float4 *xs;
    float *M, *L;
    double4_32a *far, *near;
    const int *m2lx_ptr, *m2lx_src;
    const float *pairs;
    const unsigned *pad, *flag;
    const int *p2p_ptr, *nrun;
    const int2 *runs_pr;
    float *phi, *grad;              // caller's order
    unsigned *cnt_up, *cnt_dn;      // per level: cells whose M (up) / L (down) is final
    float *mpad;                    // M rows zero-padded to whole k-blocks (tensor-core M2L), or null
    int n, ncells, nleaves, depth, c0;  // c0: first cell of level 2
    int lvl_start[FMM_MAXLEVEL + 2];
};

// work items of the batch kernels: system, kind, cell, level
enum { BATCH_P2M = 0, BATCH_M2M = 1, BATCH_L2L = 2, BATCH_L2P = 3 };

// counters written by the traversal and read back by the host
struct TravCounters {
    unsigned long long n_p2p, n_m2lx, n_next, n_m2l_implicit;
};

// CUDA events of one build and one evaluation (build: ev[0], ev[1];
// evaluation: ev[2] .. ev[12]); a handle keeps FMM_TIMING_SLOTS of them so the
// phase times of recent calls can be read back without a host sync per call
#define FMM_TIMING_SLOTS 32
struct Timers {
    cudaEvent_t ev[16] = {};
};

}  // namespace fmm

struct fmm_ctx {
    // parameters
    int64_t Nmax = 0;
    int p = 0;
    double theta = 0, cmac = 0;  // cmac = fl(theta * theta)
    int ncrit = 0;
    int precision_req = FMM_FP64;
    int engine_req = FMM_M2L_AUTO;
    // device
    int dev = 0, nsm = 0, cc_major = 0, cc_minor = 0;
    cudaStream_t stream = nullptr;  // caller's stream (or legacy default)
    cudaStream_t s2 = nullptr;      // private low-priority stream: P2P
    cudaStream_t sfar = nullptr;    // private high-priority stream: the far-field chain
    cudaStream_t work = nullptr;    // stream the far-field kernels are launched on
    cudaEvent_t ev_far = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    fmm::Timers tms[FMM_TIMING_SLOTS];
    int64_t nbuilds = 0, nevals = 0;  // successful builds and evaluations so far
    cudaEvent_t *ev_cur = nullptr;    // events of the call in progress
    int64_t launches = 0;

    // state of the last build
    bool built = false, evaluated = false;
    int64_t n = 0;
    int dtype = FMM_F64;
    bool host_mem = false;
    int precision = FMM_FP64;
    int engine_used = 0;
    int overlap = 1;  // far and near field on concurrent streams
    int lattice_extent = 0;  // largest same-level coordinate difference of existing cells
    std::vector<int> lvl_ext;  // per level: the same, -1 for an empty level
    int ncells = 0, depth = 0, nleaves = 0;
    std::vector<int> lvl_start;  // cells of level l are [lvl_start[l], lvl_start[l+1])
    int64_t n_p2p = 0, n_m2lx = 0, n_m2l_implicit = 0, n_interactions = 0;
    int ntiles_max = 0;
    int p2p_cap_hint = 0;       // near-field stencil size (P2P sources of a leaf in a uniform tree)
    bool uniform_req = true;    // full octrees take the lattice-stencil lists (fmm_set_uniform_path)
    int m2l_pool = -1;          // levels with at most this many cells pool their octants' M2L tiles (-1: 4 tiles)
    bool uniform_used = false;  // the last build did
    double ms_build = 0;

    // stencil of same-level M2L (host copy and device copy)
    int nV = 0;                 // distinct translation vectors over all octants
    std::vector<int> st_off;    // st_off[o] .. st_off[o+1]: entries of octant o; [8] .. [9]: their union
    std::vector<int> st_host;   // 4 ints per entry: vx, vy, vz (source - target), id | octant mask << 16
    fmm::DevBuf st_dev;         // int4 per entry
    int st_R = 0;               // offsets |v_k| <= st_R are in the stencil
    fmm::DevBuf rtab64, rtab32; // R_n^m(t_o), 8 child offsets, full complex storage of degree < p
    fmm::DevBuf m2m_mat, l2l_mat; // FP32 p^2 x p^2 real maps of M2M and L2L per child octant, [o][in][out]
    fmm::DevBuf ttab;           // tensor-core M2L operators (split TF32 images), per vector
    size_t ttab_stride = 0;     // bytes per vector in ttab
    int ttab_nv = -1;           // stencil vectors the operator images were made for
    fmm::DevBuf rot_tab;        // rotation M2L maps per vector ([A | B], FP32 or FP64)
    int rot_nv = -1, rot_kind = 0;  // vectors and precision (1 FP32, 2 FP64) of rot_tab
    fmm::DevBuf msplit;         // M~ split into TF32 (hi, lo) rows for the tensor-core M2L
    // tensor-core M2L on complete levels: M~ of each such level in lattice
    // order (octant bits, then z, y, x of the halved position), one TMA tensor
    // map per level (device copy and its pinned staging)
    bool lattice_req = true;    // fmm_set_m2l_lattice
    unsigned lat_levels = 0;    // bit l: level l reads its sources from the lattice copy
    long long lat_off[FMM_MAXLEVEL + 1] = {};  // float offset of level l in mlat
    fmm::DevBuf mlat, lat_maps;
    fmm::PinnedBuf lat_host;

    // workspaces
    fmm::DevBuf box;
    fmm::DevBuf x_in, q_in, w_in;       // staging of host inputs
    fmm::DevBuf keys, keys2, idx, idx2; // Morton keys and permutation (radix sort ping-pong)
    fmm::DevBuf inv;                    // inverse permutation: sorted position of each input particle
    fmm::DevBuf pcell;                  // leaf cell of each sorted particle
    fmm::DevBuf cgeo;                   // per cell: geometric centre and 1 / width (double4)
    fmm::DevBuf energy_buf;             // block sums of the weighted energy
    fmm::DevBuf hist, scan_tmp;
    fmm::DevBuf xs64, xs32, xs32lo;
    fmm::DevBuf c_level, c_anchor, c_begin, c_end, c_child, c_nchild, c_parent, c_xyz;
    fmm::DevBuf split_cnt, split_off, split_bnd;
    fmm::DevBuf leaves;
    fmm::DevBuf frontA, frontB;
    fmm::DevBuf p2p_pairs, m2lx_pairs;
    fmm::DevBuf near_dev;       // near-field stencil of the uniform fast path (int4)
    fmm::DevBuf pair_keys, pair_keys2, pair_vals, pair_vals2;
    fmm::DevBuf p2p_ptr, p2p_src, m2lx_ptr, m2lx_src, row_cnt;
    fmm::DevBuf p2p_runs, p2p_nrun;     // P2P sources merged into particle runs per target leaf
    // packed P2P of FP32 inputs: sorted particles as pair records (x0 x1 y0 y1 | z0 z1 q0 q1), each leaf
    // padded to an even count by a zero-charge copy of its last particle; pad[i] = padding before
    // particle i; the runs in pair units
    fmm::DevBuf pr_pad, pr_flag, pr_pairs, p2p_runs_pr;
    bool pr_ready = false;
    fmm::DevBuf counters;
    fmm::DevBuf lvl_desc, map_pool, hash_pool;
    fmm::DevBuf m2l_tgt, m2l_tiles, m2l_misc;
    fmm::DevBuf Mexp, Lexp;
    fmm::DevBuf far, near;
    fmm::DevBuf out_phi, out_grad;      // staging of host outputs
    fmm::DevBuf direct_part;
    fmm::PinnedBuf hpin;

    ~fmm_ctx();
};

namespace fmm {

// launch bookkeeping: every kernel launch of the library goes through this
inline void count_launch(fmm_ctx *h) { h->launches++; }
// Dynamic shared memory of a kernel beyond the 48 KB default: the attribute
// belongs to the device that is current when it is set, so it is set once per
// (kernel, device) and raised when a launch needs more (thread safe).
void ensure_smem(const void *kernel, size_t bytes);
void check_launch(const char *what);

// tree.cu
void tree_build(fmm_ctx *h, const void *x, const void *q, int64_t n, int dtype_base);
void tree_export(fmm_ctx *h, uint64_t *keys, int32_t *perm, int32_t *level, uint64_t *anchor,
                 int32_t *begin, int32_t *end, int32_t *child, int32_t *nchild, int32_t *parent,
                 int64_t *p2p_ptr, int32_t *p2p_idx, int64_t *m2l_ptr, int32_t *m2l_idx, double *box);
int64_t tree_m2l_total(fmm_ctx *h);
void morton_sort_into(const void *x, int64_t n, int dt, uint64_t *keys, int *perm, uint64_t *keys_tmp, int *perm_tmp,
                      unsigned *hist, unsigned *bsum, Box *box, int nsm, cudaStream_t s);
int m2l_tile_size(fmm_ctx *h);
void scan_exclusive_u32(fmm_ctx *h, const unsigned *in, unsigned *out, int64_t count, unsigned *total_dev,
                        cudaStream_t s);

// expansions.cu
void operators_init(fmm_ctx *h);  // R tables of M2M / L2L
void stencil_update(fmm_ctx *h);  // same-level M2L stencil for the current tree depth
// rotation-based M2L: per-degree maps into / out of the frame whose z axis is u
int rot_deg_off(int n);
int rot_map_size(int p);
void rotation_maps(int p, const double u[3], double *A, double *B);
void m2l_rotation_ref(int p, const double u[3], const double *M, double *L);
template <class T>
void m2l_rotation(fmm_ctx *h, T *L, const T *M);  // same-level M2L of all tiles by rotation
bool rotation_m2l_supported(fmm_ctx *h);           // p <= 16 (the maps of a vector fit shared memory)
int rotation_tile_rows(fmm_ctx *h);  // target cells per tile (two per warp)
// per (octant, level): how many of the octant's entries (shortest first) can
// reach a cell of that level in the current tree; written after the offsets
void stencil_levels(fmm_ctx *h, cudaStream_t s);
// device copy of the stencil: entries (int4), then 10 offsets, then per set
// (octants 0..7, union 8) and level the number of entries that can reach
const int *stencil_offsets(fmm_ctx *h);
void far_field(fmm_ctx *h);       // P2M, M2M, M2L, L2L, L2P into h->far

// batched evaluation (expansions.cu, p2p.cu): persistent kernels over work
// items of many systems; every dependency wait is bounded and reports a
// timeout in *err (bit 0) instead of hanging
void batch_up(int p, int nsm, const BatchSys *sys, const int4 *items, int nitems, int *queue, const float *m2m_mat,
              int *err, cudaStream_t s);
void batch_down(int p, int nsm, const BatchSys *sys, const int4 *items, int nitems, int *queue, const float *l2l_mat,
                int *err, cudaStream_t s);
void batch_m2lx(int p, const BatchSys *sys, const int2 *items, int nitems, cudaStream_t s);
void batch_p2p(int nsm, const BatchSys *sys, const int2 *items, int nitems, int *queue, int *err, cudaStream_t s);
void batch_zero(int p, const BatchSys *sys, int nsys, cudaStream_t s);
void batch_combine(const BatchSys *sys, int nsys, const int *blk0, int nblocks, cudaStream_t s);
void cell_geometry(fmm_ctx *h, cudaStream_t s);  // h->cgeo: centre and 1 / width of every cell

// m2l_tc.cu
void tensor_tables_init(fmm_ctx *h);
bool tensor_m2l_supported(fmm_ctx *h);
void m2l_tensor(fmm_ctx *h, float *L, const float *M);
// the same-level M2L of several systems (same p; mrow already padded to
// whole k-blocks where p^2 is not a multiple of 32) in one persistent launch
void m2l_tensor_jobs(int p, int nsm, const M2LJob *jobs_dev, int njobs, int *queue, int *err, cudaStream_t s);
M2LJob m2l_tensor_job(fmm_ctx *h, float *L, const float *M, cudaStream_t s);  // pads M if needed
// (build) which complete levels the tensor-core M2L reads through TMA tile
// loads: their lattice buffer and tensor maps
void lattice_prepare(fmm_ctx *h, cudaStream_t s);
void batch_mpad(int p, const BatchSys *sys, int nsys, cudaStream_t s);  // every system's padded M rows

// p2p.cu
void near_field(fmm_ctx *h, cudaStream_t s);  // P2P into h->near
void p2p_prepare(fmm_ctx *h, cudaStream_t s);  // pair records and pair-unit runs of the packed P2P (build)
void p2p_pairs_fill(fmm_ctx *h, cudaStream_t s);  // pair records from the sorted particles (build, new charges)
void combine_unsort(fmm_ctx *h, void *phi, void *grad);
void update_charges(fmm_ctx *h, const void *q, const void *w);
double energy(fmm_ctx *h, const void *w, const void *q, const void *phi);
void energy_adjoint(fmm_ctx *h, double gE, const void *w, const void *q, const void *phi, const void *grad,
                    const void *psi, const void *gpsi, void *dq, void *dx, void *dw);
void direct_sum(fmm_ctx *h, const double *x, const double *q, int64_t n, const int64_t *tidx, int64_t nt,
                double *phi, double *grad);

// packed real layout of an order-p expansion
__host__ __device__ inline int re_idx(int n, int m) { return n * n + (m == 0 ? 0 : 2 * m - 1); }
__host__ __device__ inline int im_idx(int n, int m) { return n * n + 2 * m; }

}  // namespace fmm

namespace fmm {

// 21-bit integer -> every third bit of a 63-bit word (bit b -> bit 3b)
__host__ __device__ inline uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__host__ __device__ inline uint64_t morton3(uint32_t x, uint32_t y, uint32_t z)
{
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// The same interleave for coordinates below 2^10 (levels <= 10), in 32-bit
// arithmetic.
__host__ __device__ inline uint32_t morton3_10(uint32_t x, uint32_t y, uint32_t z)
{
    auto sp = [](uint32_t v) {
        v &= 0x3ffu;
        v = (v | (v << 16)) & 0x030000ffu;
        v = (v | (v << 8)) & 0x0300f00fu;
        v = (v | (v << 4)) & 0x030c30c3u;
        v = (v | (v << 2)) & 0x09249249u;
        return v;
    };
    return sp(x) | (sp(y) << 1) | (sp(z) << 2);
}

// slot of a key in a table of hash_mask + 1 slots (multiplicative hashing)
__host__ __device__ inline unsigned level_hash(unsigned long long key, unsigned mask)
{
    return (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 32) & mask;
}

// Cell at lattice position (x, y, z) of level l, or -1.
__device__ inline int level_lookup(const LevelDesc &L, const int *__restrict__ map_pool,
                                   const uint64_t *__restrict__ anchor, int l, int x, int y, int z)
{
    const int side = 1 << l;
    if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) return -1;
    const uint64_t k = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
    if (L.map_off >= 0) return map_pool[L.map_off + (long long)k];
    if (L.hash) {
        // linear probing from the key's hash; the table is at most half full
        const unsigned long long key = k + 1;
        unsigned hs = level_hash(key, L.hash_mask);
        for (unsigned i = 0; i <= L.hash_mask; i++, hs = (hs + 1) & L.hash_mask) {
            const unsigned long long kk = L.hash[hs].key;
            if (kk == key) return L.hash[hs].val;
            if (kk == 0) return -1;
        }
        return -1;
    }
    const uint64_t a = k << (3 * (FMM_MAXLEVEL - l));
    int lo = L.start, hi = L.end;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (anchor[mid] < a) lo = mid + 1;
        else hi = mid;
    }
    return (lo < L.end && anchor[lo] == a) ? lo : -1;
}

}  // namespace fmm
