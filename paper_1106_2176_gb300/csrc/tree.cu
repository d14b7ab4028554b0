// Morton octree build and dual-tree interaction lists on the GPU.
//
// Sec. 2.1 of Yokota & Barba (arXiv:1106.2176) subdivides space hierarchically
// into near and far regions; Sec. 2.2 and Sec. 5 index the boxes by a Morton
// key at a prescribed maximum level and address particles through sorted
// indices with start/offset ranges. This file builds exactly that, all on the
// device and integer or correctly rounded FP64, so that keys, permutation,
// cells and lists are bit-identical to an independent CPU implementation:
//   bounding cube -> 21-bit quantisation -> 63-bit Morton keys -> stable LSD
//   radix sort -> top-down cell split (ncrit) -> level-synchronous dual
//   traversal with the theta MAC -> CSR lists.
// Same-level M2L pairs are not stored: two existing cells of one level form an
// M2L pair exactly when their lattice offset lies in the stencil of the
// target's octant (the MAC accepts them and rejects their parents), so the M2L
// kernels enumerate them through a per-level lattice lookup.
#include <algorithm>
#include <climits>
#include <cmath>

#include "fmm_internal.cuh"

namespace fmm {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
static inline unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void check_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error{FMM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

__device__ __forceinline__ unsigned long long ord_enc(double d)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ double ord_dec(unsigned long long e)
{
    unsigned long long u = (e >> 63) ? (e & 0x7fffffffffffffffull) : ~e;
    return __longlong_as_double((long long)u);
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 (three kernels; any length up to 2^31)
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024, SCAN_I = 4, SCAN_TILE = SCAN_T * SCAN_I;

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *sw, unsigned *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned s = lane < nw ? sw[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sw[lane] = s;
    }
    __syncthreads();
    unsigned base = w ? sw[w - 1] : 0u;
    if (total) *total = sw[nw - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void scan_reduce_k(const unsigned *__restrict__ in, int64_t n, unsigned *__restrict__ bsum)
{
    __shared__ unsigned sw[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; k++)
        if (base + k < n) s += in[base + k];
    unsigned tot;
    block_excl_scan(s, sw, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void scan_top_k(unsigned *bsum, int nb, unsigned *total)
{
    __shared__ unsigned sw[32];
    unsigned carry = 0;
    for (int b0 = 0; b0 < nb; b0 += SCAN_T) {
        int i = b0 + threadIdx.x;
        unsigned v = i < nb ? bsum[i] : 0u;
        unsigned tot;
        unsigned ex = block_excl_scan(v, sw, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void scan_apply_k(const unsigned *__restrict__ in, unsigned *__restrict__ out, int64_t n,
                             const unsigned *__restrict__ bsum)
{
    __shared__ unsigned sw[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    unsigned v[SCAN_I];
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; k++) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        s += v[k];
    }
    unsigned ex = block_excl_scan(s, sw, nullptr) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_I; k++) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
}

void scan_exclusive_u32(fmm_ctx *h, const unsigned *in, unsigned *out, int64_t count, unsigned *total_dev,
                        cudaStream_t s)
{
    if (count <= 0) {
        if (total_dev) FMM_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(unsigned), s));
        return;
    }
    int nb = (int)nblocks(count, SCAN_TILE);
    h->scan_tmp.ensure(sizeof(unsigned) * (size_t)(nb + 1));
    unsigned *bsum = h->scan_tmp.as<unsigned>();
    scan_reduce_k<<<nb, SCAN_T, 0, s>>>(in, count, bsum);
    count_launch(h);
    scan_top_k<<<1, SCAN_T, 0, s>>>(bsum, nb, total_dev);
    count_launch(h);
    scan_apply_k<<<nb, SCAN_T, 0, s>>>(in, out, count, bsum);
    count_launch(h);
    check_launch("scan");
}

// ---------------------------------------------------------------------------
// bounding cube and Morton keys
// ---------------------------------------------------------------------------
__global__ void box_init_k(Box *b)
{
    for (int k = 0; k < 3; k++) {
        b->enc_lo[k] = ~0ull;
        b->enc_hi[k] = 0ull;
    }
    b->nonfinite = 0;
}

// FP32 -> FP64 without flushing subnormal inputs (the library is built with
// flush-to-zero for its FP32 arithmetic; the box and the keys use every
// input value exactly)
__device__ __forceinline__ double f32_to_f64_exact(float v)
{
    double d;
    asm("cvt.f64.f32 %0, %1;" : "=d"(d) : "f"(v));
    return d;
}
__device__ __forceinline__ double to_f64_exact(float v) { return f32_to_f64_exact(v); }
__device__ __forceinline__ double to_f64_exact(double v) { return v; }

template <class T>
__global__ void bbox_k(const T *__restrict__ x, int64_t n, Box *b)
{
    // FP32 input: each thread's extremes as order-preserving integer
    // encodings of the float bits (exact, subnormals included, and off
    // GB300's slow FP64 pipe), converted to FP64 once; FP64 input in FP64
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    if constexpr (sizeof(T) == 4) {
        // (no finite value encodes to 0xffffffff or to 0: the initial values mark "none seen")
        unsigned elo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, ehi[3] = {0u, 0u, 0u};
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const unsigned u = __float_as_uint((float)x[3 * i + k]);
                if ((u & 0x7f800000u) == 0x7f800000u) bad = 1;
                else {
                    const unsigned e = (u >> 31) ? ~u : (u | 0x80000000u);
                    elo[k] = min(elo[k], e);
                    ehi[k] = max(ehi[k], e);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 3; k++)
            if (elo[k] != 0xffffffffu) {
                const unsigned a = (elo[k] >> 31) ? (elo[k] & 0x7fffffffu) : ~elo[k];
                const unsigned c = (ehi[k] >> 31) ? (ehi[k] & 0x7fffffffu) : ~ehi[k];
                lo[k] = f32_to_f64_exact(__uint_as_float(a));
                hi[k] = f32_to_f64_exact(__uint_as_float(c));
            }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const double v = (double)x[3 * i + k];
                if (!isfinite(v)) bad = 1;
                else {
                    lo[k] = fmin(lo[k], v);
                    hi[k] = fmax(hi[k], v);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; k++)
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 3; k++) {
            if (lo[k] <= hi[k]) {
                atomicMin(&b->enc_lo[k], ord_enc(lo[k]));
                atomicMax(&b->enc_hi[k], ord_enc(hi[k]));
            }
        }
        if (bad) atomicOr(&b->nonfinite, 1);
    }
}

// Root cube from the bounding box, all in correctly rounded FP64:
// c = (lo + hi) / 2, R0 = max half extent (1 if 0), origin = c - R0,
// s = 2^21 / (2 R0), h = 2 R0 / 2^21.
__global__ void box_final_k(Box *b)
{
    double R0 = 0.0, c[3];
    for (int k = 0; k < 3; k++) {
        double lo = ord_dec(b->enc_lo[k]), hi = ord_dec(b->enc_hi[k]);
        c[k] = __dmul_rn(__dadd_rn(lo, hi), 0.5);
        double half = __dmul_rn(__dsub_rn(hi, lo), 0.5);
        if (half > R0) R0 = half;
    }
    if (R0 == 0.0) R0 = 1.0;
    for (int k = 0; k < 3; k++) b->origin[k] = __dsub_rn(c[k], R0);
    b->R0 = R0;
    b->s = __ddiv_rn(2097152.0, __dmul_rn(2.0, R0));
    b->h = __ddiv_rn(__dmul_rn(2.0, R0), 2097152.0);
}

// i_k = clamp(floor((x_k - origin_k) * s), 0, 2^21 - 1); key interleaves
// x, y, z bits with x lowest.
template <class T>
__global__ void keys_k(const T *__restrict__ x, int64_t n, const Box *__restrict__ b, uint64_t *__restrict__ keys,
                       int *__restrict__ idx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t ic[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double v = to_f64_exact(x[3 * i + k]);
        // floor to an integer in one conversion (saturating), clamped as an
        // integer: the same value as floor, clamp and cast in FP64, with half
        // the FP64 instructions
        const int f = __double2int_rd(__dmul_rn(__dsub_rn(v, b->origin[k]), b->s));
        ic[k] = (uint32_t)min(max(f, 0), 2097151);
    }
    keys[i] = morton3(ic[0], ic[1], ic[2]);
    idx[i] = (int)i;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of 64-bit keys (8-bit digits) with int32 values
// ---------------------------------------------------------------------------
constexpr int RS_T = 256, RS_W = RS_T / 32, RS_R = 16, RS_TILE = RS_T * RS_R;  // 4096 keys per tile

__global__ void __launch_bounds__(RS_T) rs_hist_k(const uint64_t *__restrict__ keys, int n, int shift,
                                                   unsigned *__restrict__ hist, int ntiles)
{
    __shared__ unsigned hcount[256];
    hcount[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_T) {
        int g = base + i;
        if (g < n) atomicAdd(&hcount[(unsigned)(keys[g] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = hcount[threadIdx.x];
}

// Each warp ranks its 512 consecutive keys in 16 rounds of 32 (match_any on
// the digit), so the rank of a key among equal digits follows input order;
// the tile is staged in shared memory in digit order and written out in runs.
template <bool VALS>
__global__ void __launch_bounds__(RS_T) rs_scatter_k(const uint64_t *__restrict__ kin, const int *__restrict__ vin,
                                                      uint64_t *__restrict__ kout, int *__restrict__ vout, int n,
                                                      int shift, const unsigned *__restrict__ offs, int ntiles)
{
    extern __shared__ unsigned char smem_raw[];
    uint64_t *skey = reinterpret_cast<uint64_t *>(smem_raw);               // RS_TILE
    int *sval = reinterpret_cast<int *>(skey + RS_TILE);                   // RS_TILE
    unsigned *wcnt = reinterpret_cast<unsigned *>(sval + RS_TILE);         // RS_W * 256
    unsigned *dstart = wcnt + RS_W * 256;                                  // 256
    unsigned *goff = dstart + 256;                                         // 256
    unsigned *sw = goff + 256;                                             // 32

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int base = blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_W * 256; i += RS_T) wcnt[i] = 0;
    goff[threadIdx.x] = offs[threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();

    const unsigned lt = (1u << lane) - 1u;
    uint64_t k[RS_R];
    int v[RS_R];
    unsigned rank[RS_R];
#pragma unroll
    for (int r = 0; r < RS_R; r++) {
        int i = base + w * (32 * RS_R) + r * 32 + lane;
        bool ok = i < n;
        k[r] = ok ? kin[i] : ~0ull;
        v[r] = (VALS && ok) ? vin[i] : 0;
        unsigned d = (unsigned)(k[r] >> shift) & 255u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned c = wcnt[w * 256 + d];
        rank[r] = c + __popc(peers & lt);
        __syncwarp();
        if (lane == __ffs(peers) - 1) wcnt[w * 256 + d] = c + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps and the tile total
    {
        unsigned run = 0;
        for (int ww = 0; ww < RS_W; ww++) {
            unsigned c = wcnt[ww * 256 + threadIdx.x];
            wcnt[ww * 256 + threadIdx.x] = run;
            run += c;
        }
        unsigned ex = block_excl_scan(run, sw, nullptr);
        dstart[threadIdx.x] = ex;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_R; r++) {
        unsigned d = (unsigned)(k[r] >> shift) & 255u;
        unsigned pos = dstart[d] + wcnt[w * 256 + d] + rank[r];
        skey[pos] = k[r];
        if (VALS) sval[pos] = v[r];
    }
    __syncthreads();
    const int nvalid = min(RS_TILE, n - base);
    for (int j = threadIdx.x; j < nvalid; j += RS_T) {
        uint64_t kk = skey[j];
        unsigned d = (unsigned)(kk >> shift) & 255u;
        unsigned g = goff[d] + (unsigned)j - dstart[d];
        kout[g] = kk;
        if (VALS) vout[g] = sval[j];
    }
}

static size_t rs_smem() { return (size_t)RS_TILE * 12 + (size_t)(RS_W * 256 + 256 + 256 + 32) * 4; }

// Sorts by the low `bits` bits of the keys. Returns true when the result sits
// in (kt, vt) rather than (k, v).
static bool radix_sort(fmm_ctx *h, uint64_t *k, int *v, uint64_t *kt, int *vt, int64_t n64, int bits,
                       cudaStream_t s)
{
    if (n64 <= 1 || bits <= 0) return false;
    if (n64 > 0x7fffffffLL) throw Error{FMM_EINVAL, "radix sort: too many keys"};
    const int n = (int)n64;
    const int ntiles = (int)nblocks(n, RS_TILE);
    h->hist.ensure(sizeof(unsigned) * (size_t)256 * ntiles);
    unsigned *hist = h->hist.as<unsigned>();
    ensure_smem((const void *)rs_scatter_k<true>, rs_smem());
    ensure_smem((const void *)rs_scatter_k<false>, rs_smem());
    bool swapped = false;
    for (int shift = 0; shift < bits; shift += 8) {
        rs_hist_k<<<ntiles, RS_T, 0, s>>>(k, n, shift, hist, ntiles);
        count_launch(h);
        scan_exclusive_u32(h, hist, hist, (int64_t)256 * ntiles, nullptr, s);
        if (v) rs_scatter_k<true><<<ntiles, RS_T, rs_smem(), s>>>(k, v, kt, vt, n, shift, hist, ntiles);
        else rs_scatter_k<false><<<ntiles, RS_T, rs_smem(), s>>>(k, nullptr, kt, nullptr, n, shift, hist, ntiles);
        count_launch(h);
        check_launch("radix sort");
        std::swap(k, kt);
        std::swap(v, vt);
        swapped = !swapped;
    }
    return swapped;
}

// Sorted particles (x, y, z, q). For the mixed path the FP32 copy holds the
// rounded coordinates, and xs32lo the FP32 rounding of the remainder x - hi
// (zero for FP32 inputs), so that a near-field difference can be formed as
// (hi_i - hi_j) + (lo_i - lo_j) without the rounding of the positions.
// Morton keys and their stable sort into caller-provided buffers, with every
// temporary taken from caller-provided scratch (no allocation): the first
// stages of the tree build, for the allocation-free entry point.
//   keys[n], perm[n]         results (sorted keys, input index of each)
//   keys_tmp[n], perm_tmp[n] ping-pong buffers
//   hist[256 * ceil(n / 4096)], bsum[ceil(256 * ceil(n / 4096) / 4096) + 1]
//   box                      root-cube scratch
void morton_sort_into(const void *x, int64_t n64, int dt, uint64_t *keys, int *perm, uint64_t *keys_tmp, int *perm_tmp,
                      unsigned *hist, unsigned *bsum, Box *box, int nsm, cudaStream_t s)
{
    const int n = (int)n64;
    const int TB = 256;
    box_init_k<<<1, 1, 0, s>>>(box);
    const int bb_blocks = std::max(1, std::min((int)nblocks(n, TB), nsm * 8));
    if (dt == FMM_F64) {
        bbox_k<double><<<bb_blocks, TB, 0, s>>>((const double *)x, n, box);
        box_final_k<<<1, 1, 0, s>>>(box);
        keys_k<double><<<nblocks(n, TB), TB, 0, s>>>((const double *)x, n, box, keys, perm);
    } else {
        bbox_k<float><<<bb_blocks, TB, 0, s>>>((const float *)x, n, box);
        box_final_k<<<1, 1, 0, s>>>(box);
        keys_k<float><<<nblocks(n, TB), TB, 0, s>>>((const float *)x, n, box, keys, perm);
    }
    check_launch("keys");
    if (n <= 1) return;
    FMM_CUDA_TRY(cudaFuncSetAttribute(rs_scatter_k<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_smem()));
    const int ntiles = (int)nblocks(n, RS_TILE);
    const int64_t nh = (int64_t)256 * ntiles;
    const int nb = (int)nblocks(nh, SCAN_TILE);
    uint64_t *k = keys, *kt = keys_tmp;
    int *v = perm, *vt = perm_tmp;
    for (int shift = 0; shift < 63; shift += 8) {  // 8 passes: the result ends in keys / perm
        rs_hist_k<<<ntiles, RS_T, 0, s>>>(k, n, shift, hist, ntiles);
        scan_reduce_k<<<nb, SCAN_T, 0, s>>>(hist, nh, bsum);
        scan_top_k<<<1, SCAN_T, 0, s>>>(bsum, nb, nullptr);
        scan_apply_k<<<nb, SCAN_T, 0, s>>>(hist, hist, nh, bsum);
        rs_scatter_k<true><<<ntiles, RS_T, rs_smem(), s>>>(k, v, kt, vt, n, shift, hist, ntiles);
        check_launch("radix sort");
        std::swap(k, kt);
        std::swap(v, vt);
    }
}

template <class T>
__global__ void gather_k(const T *__restrict__ x, const T *__restrict__ q, const int *__restrict__ idx, int64_t n,
                         double4_32a *__restrict__ xs64, float4 *__restrict__ xs32, float4 *__restrict__ xs32lo,
                         int *__restrict__ inv)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = idx[i];
    inv[j] = (int)i;
    const double a = to_f64_exact(x[3 * (int64_t)j]), b = to_f64_exact(x[3 * (int64_t)j + 1]),
                 c = to_f64_exact(x[3 * (int64_t)j + 2]);
    const double d = to_f64_exact(q[j]);
    if (xs64) xs64[i] = make_double4_32a(a, b, c, d);
    if (xs32) {
        const float ha = (float)a, hb = (float)b, hc = (float)c;
        xs32[i] = make_float4(ha, hb, hc, (float)d);
        if (xs32lo) xs32lo[i] = make_float4((float)(a - ha), (float)(b - hb), (float)(c - hc), 0.f);
    }
}

// ---------------------------------------------------------------------------
// cells: a cell of level l < 21 with more than ncrit particles splits into its
// non-empty octants, ascending octant order, numbered breadth first
// ---------------------------------------------------------------------------
__global__ void root_k(int n, int *level, uint64_t *anchor, int *begin, int *end, int *child, int *nchild,
                       int *parent, int4 *xyz)
{
    level[0] = 0;
    anchor[0] = 0;
    begin[0] = 0;
    end[0] = n;
    child[0] = -1;
    nchild[0] = 0;
    parent[0] = -1;
    xyz[0] = make_int4(0, 0, 0, 0);
}

__global__ void split_count_k(int ls, int le, int l, int ncrit, const uint64_t *__restrict__ keys,
                              const int *__restrict__ begin, const int *__restrict__ end, unsigned *__restrict__ cnt,
                              int *__restrict__ bnd)
{
    int c = ls + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    int b = begin[c], e = end[c];
    unsigned nc = 0;
    int *bb = bnd + (size_t)(c - ls) * 9;
    if (l < FMM_MAXLEVEL && e - b > ncrit) {
        const int shift = 3 * (FMM_MAXLEVEL - 1 - l);
        bb[0] = b;
        int lo = b;
        for (int o = 1; o < 8; o++) {
            int L = lo, H = e;  // first index with digit >= o
            while (L < H) {
                int mid = (L + H) >> 1;
                if ((int)((keys[mid] >> shift) & 7u) < o) L = mid + 1;
                else H = mid;
            }
            bb[o] = L;
            lo = L;
        }
        bb[8] = e;
        for (int o = 0; o < 8; o++) nc += bb[o + 1] > bb[o];
    }
    cnt[c - ls] = nc;
}

__global__ void split_write_k(int ls, int le, int l, const unsigned *__restrict__ cnt, const unsigned *__restrict__ off,
                              const int *__restrict__ bnd, int *level, uint64_t *anchor, int *begin, int *end,
                              int *child, int *nchild, int *parent, int4 *xyz)
{
    int c = ls + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    unsigned nc = cnt[c - ls];
    nchild[c] = (int)nc;
    child[c] = nc ? le + (int)off[c - ls] : -1;
    if (!nc) return;
    const int *bb = bnd + (size_t)(c - ls) * 9;
    const int shift = 3 * (FMM_MAXLEVEL - 1 - l);
    const int bit = FMM_MAXLEVEL - 1 - l;
    const int4 pxyz = xyz[c];
    const uint64_t pa = anchor[c];
    int k = le + (int)off[c - ls];
    for (int o = 0; o < 8; o++) {
        if (bb[o + 1] <= bb[o]) continue;
        level[k] = l + 1;
        anchor[k] = pa | ((uint64_t)o << shift);
        begin[k] = bb[o];
        end[k] = bb[o + 1];
        child[k] = -1;
        nchild[k] = 0;
        parent[k] = c;
        xyz[k] = make_int4(pxyz.x | ((o & 1) << bit), pxyz.y | (((o >> 1) & 1) << bit), pxyz.z | (((o >> 2) & 1) << bit),
                           l + 1);
        k++;
    }
}

// ---------------------------------------------------------------------------
// dual traversal, one level of the pair frontier per launch
// ---------------------------------------------------------------------------

// Multipole acceptance in integer half-grid units: the box of level l is
// W = 2^(21-l) grid units wide, its centre 2*anchor + W half units, its half
// diagonal sqrt(3) W. Accept iff 3 (W_A + W_B)^2 < fl(theta^2 d^2).
__device__ __forceinline__ bool mac_accept(int4 a, int4 b, double c)
{
    const long long WA = 1LL << (FMM_MAXLEVEL - a.w), WB = 1LL << (FMM_MAXLEVEL - b.w);
    const long long dx = 2LL * (a.x - b.x) + (WA - WB);
    const long long dy = 2LL * (a.y - b.y) + (WA - WB);
    const long long dz = 2LL * (a.z - b.z) + (WA - WB);
    const long long d2 = dx * dx + dy * dy + dz * dz;
    const double lhs = __dmul_rn(3.0, (double)((WA + WB) * (WA + WB)));
    const double rhs = __dmul_rn(c, (double)d2);
    return lhs < rhs;
}

// The same test for two cells of one level: with W_A = W_B = W both sides
// carry the exact factor 4 W^2, so it reduces to 3 < fl(theta^2 |v|^2), v the
// offset in cell units, and by monotone rounding to |v|^2 >= K0 with K0 the
// first integer that passes (computed on the host with the same FP64 multiply).
__device__ __forceinline__ bool mac_accept_same(int4 a, int4 b, long long K0)
{
    const int sh = FMM_MAXLEVEL - a.w;
    const long long vx = (b.x - a.x) >> sh, vy = (b.y - a.y) >> sh, vz = (b.z - a.z) >> sh;
    return vx * vx + vy * vy + vz * vz >= K0;
}

// warp-aggregated reservation of `cnt` slots in a global counter
__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long *ctr, unsigned cnt)
{
    const int lane = threadIdx.x & 31;
    unsigned x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    unsigned long long base = 0;
    if (lane == 31 && x) base = atomicAdd(ctr, (unsigned long long)x);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + (x - cnt);
}

// Per level, the smallest and largest lattice coordinate of the existing
// cells (ext[0..66): minima, level-major x y z; ext[66..132): maxima). Lanes
// of one level reduce in the warp first; cells are level-contiguous.
__global__ void extent_k(int nc, const int4 *__restrict__ xyz, int *__restrict__ ext)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = i < nc;
    const int4 a = in ? xyz[i] : make_int4(0, 0, 0, 0);
    const int l = in ? a.w : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, l);
    if (!in) return;
    const int sh = FMM_MAXLEVEL - l;
    const int x = a.x >> sh, y = a.y >> sh, z = a.z >> sh;
    const int mnx = __reduce_min_sync(grp, x), mny = __reduce_min_sync(grp, y), mnz = __reduce_min_sync(grp, z);
    const int mxx = __reduce_max_sync(grp, x), mxy = __reduce_max_sync(grp, y), mxz = __reduce_max_sync(grp, z);
    if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) {
        int *mn = ext + 3 * l, *mx = ext + 3 * (FMM_MAXLEVEL + 1) + 3 * l;
        atomicMin(mn, mnx);
        atomicMin(mn + 1, mny);
        atomicMin(mn + 2, mnz);
        atomicMax(mx, mxx);
        atomicMax(mx + 1, mxy);
        atomicMax(mx + 2, mxz);
    }
}

// One thread per (frontier pair, slot): the pair (A, B) expands into at most
// 8 x 8 child pairs; slot k takes child a = child[A] + k of A (or A itself)
// against the children of B (or B itself), at most 8 pairs, classified in
// registers and written after one warp-aggregated reservation per list.
__global__ void __launch_bounds__(256) expand_k(const int2 *__restrict__ F, unsigned nF, const int4 *__restrict__ xyz,
                                                const int *__restrict__ child, const int *__restrict__ nchild, double cm,
                                                long long K0,
                                                int2 *__restrict__ p2p, unsigned long long cap_p2p,
                                                int2 *__restrict__ m2lx, unsigned long long cap_m2lx,
                                                int2 *__restrict__ next, unsigned long long cap_next,
                                                TravCounters *ctr)
{
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned i = (unsigned)(t >> 3), slot = (unsigned)(t & 7);
    int a = -1, b0 = 0, nb = 0;
    if (i < nF) {
        const int2 pr = F[i];
        const int A = pr.x, B = pr.y;
        const int ncA = nchild[A], ncB = nchild[B];
        const int lA = xyz[A].w, lB = xyz[B].w;
        const bool la = ncA == 0, lb = ncB == 0;
        if (!la && (lb || lA < lB)) {  // split A only
            if ((int)slot < ncA) { a = child[A] + slot; b0 = B; nb = 1; }
        } else if (!lb && (la || lB < lA)) {  // split B only
            if (slot == 0) { a = A; b0 = child[B]; nb = ncB; }
        } else {  // both, same level
            if ((int)slot < ncA) { a = child[A] + slot; b0 = child[B]; nb = ncB; }
        }
    }
    unsigned mP = 0, mX = 0, mN = 0, cI = 0;
    if (a >= 0) {
        const int4 xa = xyz[a];
        const bool leafa = nchild[a] == 0;
        for (int k = 0; k < nb; k++) {
            const int b = b0 + k;
            const int4 xb = xyz[b];
            if (xa.w == xb.w ? mac_accept_same(xa, xb, K0) : mac_accept(xa, xb, cm)) {
                if (xa.w == xb.w) cI++;
                else mX |= 1u << k;
            } else if (leafa && nchild[b] == 0) mP |= 1u << k;
            else mN |= 1u << k;
        }
    }
    unsigned long long oP = warp_reserve(&ctr->n_p2p, __popc(mP));
    unsigned long long oX = warp_reserve(&ctr->n_m2lx, __popc(mX));
    unsigned long long oN = warp_reserve(&ctr->n_next, __popc(mN));
    warp_reserve(&ctr->n_m2l_implicit, cI);
    for (; mP; mP &= mP - 1, oP++)
        if (oP < cap_p2p) p2p[oP] = make_int2(a, b0 + __ffs(mP) - 1);
    for (; mX; mX &= mX - 1, oX++)
        if (oX < cap_m2lx) m2lx[oX] = make_int2(a, b0 + __ffs(mX) - 1);
    for (; mN; mN &= mN - 1, oN++)
        if (oN < cap_next) next[oN] = make_int2(a, b0 + __ffs(mN) - 1);
}

// ---------------------------------------------------------------------------
// pair lists -> CSR (sorted by target, then source)
// ---------------------------------------------------------------------------
__global__ void pair_keys_k(const int2 *__restrict__ pr, int64_t np, int bs, uint64_t *__restrict__ keys)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    int2 v = pr[i];
    keys[i] = ((uint64_t)(unsigned)v.x << bs) | (uint64_t)(unsigned)v.y;
}

__global__ void pair_rows_k(const uint64_t *__restrict__ keys, int64_t np, int bs, unsigned *__restrict__ rowcnt,
                            int *__restrict__ src)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    uint64_t k = keys[i];
    src[i] = (int)(k & ((1ull << bs) - 1));
    const int row = (int)(k >> bs);
    const unsigned same = __match_any_sync(__activemask(), row);
    if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&rowcnt[row], (unsigned)__popc(same));
}

__global__ void interactions_k(const int *__restrict__ ptr, const int *__restrict__ src, const int *__restrict__ begin,
                               const int *__restrict__ end, int nc, unsigned long long *out)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long s = 0;
    if (c < nc) {
        long long na = end[c] - begin[c];
        for (int k = ptr[c]; k < ptr[c + 1]; k++) {
            int b = src[k];
            s += (unsigned long long)(na * (long long)(end[b] - begin[b]));
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// P2P source leaves of a target leaf that are adjacent in the sorted particle
// order are merged into runs [begin, end); runs of leaf A are stored at
// [ptr[A], ptr[A] + nrun[A]) of the run array (never more runs than leaves).
__global__ void p2p_runs_k(int nleaves, const int *__restrict__ leaves, const int *__restrict__ ptr,
                           const int *__restrict__ src, const int *__restrict__ begin, const int *__restrict__ end,
                           int2 *__restrict__ runs, int *__restrict__ nrun)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaves) return;
    const int A = leaves[i];
    int k = ptr[A], o = ptr[A];
    const int k1 = ptr[A + 1];
    while (k < k1) {
        int b = begin[src[k]], e = end[src[k]];
        k++;
        while (k < k1 && begin[src[k]] == e) {
            e = end[src[k]];
            k++;
        }
        runs[o++] = make_int2(b, e);
    }
    nrun[A] = o - ptr[A];
}

// (target, source) pairs -> CSR rows without a global sort: rows are counted
// and filled with warp-aggregated atomics, then each row is put in ascending
// source order by exact ranks (sources of a row are distinct).
__global__ void row_count_k(const int2 *__restrict__ pr, int64_t np, unsigned *__restrict__ cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int a = pr[i].x;
    const unsigned act = __activemask();
    const unsigned same = __match_any_sync(act, a);
    if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&cnt[a], (unsigned)__popc(same));
}

__global__ void row_fill_k(const int2 *__restrict__ pr, int64_t np, const int *__restrict__ ptr, unsigned *__restrict__ cur,
                           int *__restrict__ src)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int2 v = pr[i];
    const unsigned act = __activemask();
    const unsigned same = __match_any_sync(act, v.x);
    const int lane = threadIdx.x & 31, leader = __ffs(same) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&cur[v.x], (unsigned)__popc(same));
    base = __shfl_sync(same, base, leader);
    const unsigned rank = __popc(same & ((1u << lane) - 1));
    src[ptr[v.x] + base + rank] = v.y;
}

__global__ void row_max_k(int nc, const unsigned *__restrict__ cnt, unsigned *__restrict__ mx)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned v = c < nc ? cnt[c] : 0u;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(mx, v);
}

constexpr int ROW_SORT_WARPS = 8, ROW_SORT_CAP = 1024;

// Ascending bitonic sort of 256 keys held by one warp, lane l holding keys
// 8 l .. 8 l + 7: partners 8 or more apart are exchanged with shuffles, the
// others inside the lane's registers.
__device__ __forceinline__ void warp_bitonic256(int (&v)[8], int lane)
{
#pragma unroll
    for (int k = 2; k <= 256; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 8) {
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    const int i = lane * 8 + r;
                    const int y = __shfl_xor_sync(0xffffffffu, v[r], j >> 3);
                    const bool up = (i & k) == 0, low = (i & j) == 0;
                    v[r] = low == up ? min(v[r], y) : max(v[r], y);
                }
            } else {
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    if (r & j) continue;
                    const bool up = ((lane * 8 + r) & k) == 0;
                    const int a = v[r], b = v[r | j];
                    v[r] = up ? min(a, b) : max(a, b);
                    v[r | j] = up ? max(a, b) : min(a, b);
                }
            }
        }
    }
}

// Each CSR row in ascending order, one warp per row: rows of up to 256
// entries by a bitonic sort in registers, longer ones (up to ROW_SORT_CAP)
// by exact ranks in shared memory.
__global__ void __launch_bounds__(32 * ROW_SORT_WARPS) row_sort_k(int nc, const int *__restrict__ ptr, int *__restrict__ src)
{
    __shared__ int sh[ROW_SORT_WARPS][ROW_SORT_CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r = blockIdx.x * ROW_SORT_WARPS + w;
    if (r >= nc) return;
    const int b = ptr[r], len = ptr[r + 1] - b;
    if (len <= 1 || len > ROW_SORT_CAP) return;
    if (len <= 256) {
        int v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = lane * 8 + k < len ? src[b + lane * 8 + k] : INT_MAX;
        warp_bitonic256(v, lane);
#pragma unroll
        for (int k = 0; k < 8; k++)
            if (lane * 8 + k < len) src[b + lane * 8 + k] = v[k];
        return;
    }
    int *row = sh[w];
    for (int k = lane; k < len; k += 32) row[k] = src[b + k];
    __syncwarp();
    for (int k = lane; k < len; k += 32) {
        const int e = row[k];
        int rank = 0;
        for (int t = 0; t < len; t++) rank += row[t] < e;
        src[b + rank] = e;
    }
}

// ---------------------------------------------------------------------------
// uniform-tree fast path: on a full octree (every leaf on level L, every level
// full) the traversal's P2P lists are the near-field lattice stencil of level
// L, cut at the lattice boundary; cell id = first cell of level L + Morton
// index of the lattice position.  The traversal reaches a pair of leaves only
// if every pair of their ancestors was rejected; that holds for every near
// pair: theta < 1 gives K0 >= 4, and a child offset with |v|^2 <= K0 - 1 has a
// parent offset with |u_d| <= (|v_d| + 1) / 2, so
// |u|^2 <= (|v|^2 + 2 sqrt(3) |v| + 3) / 4 < K0.
// ---------------------------------------------------------------------------
// write = false: row counts into cnt[c]; write = true: the rows at ptr[c]
__global__ void near_rows_k(int ls, int le, int L, const int4 *__restrict__ xyz, const int4 *__restrict__ near,
                            int nnear, unsigned *__restrict__ cnt, const int *__restrict__ ptr,
                            int *__restrict__ src, bool write)
{
    const int c = ls + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    const int sh = FMM_MAXLEVEL - L, side = 1 << L;
    const int4 a = xyz[c];
    const int px = a.x >> sh, py = a.y >> sh, pz = a.z >> sh;
    int k = 0, base = write ? ptr[c] : 0;
    for (int e = 0; e < nnear; e++) {
        const int4 v = near[e];
        const int qx = px + v.x, qy = py + v.y, qz = pz + v.z;
        if (qx < 0 || qy < 0 || qz < 0 || qx >= side || qy >= side || qz >= side) continue;
        if (write) src[base + k] = ls + (int)morton3((uint32_t)qx, (uint32_t)qy, (uint32_t)qz);
        k++;
    }
    if (!write) cnt[c] = (unsigned)k;
}

static int bits_for(int64_t v)
{
    int b = 1;
    while ((1LL << b) <= v) b++;
    return b;
}

// Sort np (target, source) pairs into CSR rows over ncells cells.
static void pairs_to_csr(fmm_ctx *h, const int2 *pairs, int64_t np, DevBuf &ptr, DevBuf &src, cudaStream_t s)
{
    const int nc = h->ncells;
    ptr.ensure(sizeof(int) * (size_t)(nc + 1));
    src.ensure(sizeof(int) * (size_t)std::max<int64_t>(np, 1));
    h->row_cnt.ensure(sizeof(unsigned) * (size_t)(nc + 1));
    FMM_CUDA_TRY(cudaMemsetAsync(h->row_cnt.p, 0, sizeof(unsigned) * (size_t)(nc + 1), s));
    if (np > 0) {
        row_count_k<<<nblocks(np, 256), 256, 0, s>>>(pairs, np, h->row_cnt.as<unsigned>());
        count_launch(h);
        // longest row: rows that fit the per-warp sort are filled and ranked
        // in place, otherwise the pairs go through a global sort
        unsigned *dmax = reinterpret_cast<unsigned *>(h->counters.as<char>() + sizeof(TravCounters) + 32);
        FMM_CUDA_TRY(cudaMemsetAsync(dmax, 0, sizeof(unsigned), s));
        row_max_k<<<nblocks(nc, 256), 256, 0, s>>>(nc, h->row_cnt.as<unsigned>(), dmax);
        count_launch(h);
        unsigned *hp = h->hpin.as<unsigned>();
        FMM_CUDA_TRY(cudaMemcpyAsync(hp, dmax, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        if (*hp <= (unsigned)ROW_SORT_CAP) {
            scan_exclusive_u32(h, h->row_cnt.as<unsigned>(), reinterpret_cast<unsigned *>(ptr.as<int>()), nc + 1, nullptr, s);
            FMM_CUDA_TRY(cudaMemsetAsync(h->row_cnt.p, 0, sizeof(unsigned) * (size_t)(nc + 1), s));
            row_fill_k<<<nblocks(np, 256), 256, 0, s>>>(pairs, np, ptr.as<int>(), h->row_cnt.as<unsigned>(), src.as<int>());
            count_launch(h);
            row_sort_k<<<nblocks(nc, ROW_SORT_WARPS), 32 * ROW_SORT_WARPS, 0, s>>>(nc, ptr.as<int>(), src.as<int>());
            count_launch(h);
            check_launch("pairs to csr");
            return;
        }
        FMM_CUDA_TRY(cudaMemsetAsync(h->row_cnt.p, 0, sizeof(unsigned) * (size_t)(nc + 1), s));
        const int bs = bits_for(nc - 1);
        h->pair_keys.ensure(sizeof(uint64_t) * (size_t)np);
        h->pair_keys2.ensure(sizeof(uint64_t) * (size_t)np);
        uint64_t *k1 = h->pair_keys.as<uint64_t>(), *k2 = h->pair_keys2.as<uint64_t>();
        pair_keys_k<<<nblocks(np, 256), 256, 0, s>>>(pairs, np, bs, k1);
        count_launch(h);
        bool sw = radix_sort(h, k1, nullptr, k2, nullptr, np, 2 * bs, s);
        const uint64_t *ks = sw ? k2 : k1;
        pair_rows_k<<<nblocks(np, 256), 256, 0, s>>>(ks, np, bs, h->row_cnt.as<unsigned>(), src.as<int>());
        count_launch(h);
        check_launch("pairs to csr");
    }
    scan_exclusive_u32(h, h->row_cnt.as<unsigned>(), reinterpret_cast<unsigned *>(ptr.as<int>()), nc + 1, nullptr, s);
}

// ---------------------------------------------------------------------------
// per-level lattice maps and M2L target tiles
// ---------------------------------------------------------------------------
__global__ void map_fill_k(int ls, int le, int l, const uint64_t *__restrict__ anchor, int *__restrict__ map)
{
    int c = ls + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    map[anchor[c] >> (3 * (FMM_MAXLEVEL - l))] = c;
}

// the cells of a level without a dense map into its open-addressed table
// (linear probing; at most half full, so every insertion finds a slot)
__global__ void hash_fill_k(int ls, int le, int l, const uint64_t *__restrict__ anchor, HashSlot *__restrict__ tab,
                            unsigned mask)
{
    int c = ls + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    const unsigned long long key = (anchor[c] >> (3 * (FMM_MAXLEVEL - l))) + 1ull;
    unsigned hs = level_hash(key, mask);
    for (unsigned i = 0; i <= mask; i++, hs = (hs + 1) & mask) {
        const unsigned long long prev = atomicCAS(&tab[hs].key, 0ull, key);
        if (prev == 0ull || prev == key) {
            tab[hs].val = c;
            return;
        }
    }
}

__global__ void oct_count_k(int c0, int nc, const int *__restrict__ level, const uint64_t *__restrict__ anchor,
                            unsigned *__restrict__ grp)
{
    int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int l = level[c];
    int o = (int)((anchor[c] >> (3 * (FMM_MAXLEVEL - l))) & 7u);
    atomicAdd(&grp[l * 8 + o], 1u);
}

// One thread: group offsets and tile descriptors, levels 2..depth.
// Levels with at most pool_max cells would leave the tiles of their octant
// groups mostly empty: their cells (every octant) are pooled, level by level,
// at the front of the target list and cut into tiles of octant 8, whose
// level is the largest level among their cells. Within a denser level the
// tiles of the 8 octant groups are interleaved (tile k of octant 0, tile k of
// octant 1, ...), so that tiles running at the same time cover one compact
// region and share sources in L2.
__global__ void tiles_k(int depth, int tile, int pool_max, const unsigned *__restrict__ grp,
                        unsigned *__restrict__ goff, M2LTile *__restrict__ tiles, int *__restrict__ ntiles)
{
    unsigned run = 0;
    int nt = 0;
    auto level_cells = [&](int l) {
        unsigned c = 0;
        for (int o = 0; o < 8; o++) c += grp[l * 8 + o];
        return c;
    };
    for (int l = 2; l <= depth; l++) {
        if (level_cells(l) > (unsigned)pool_max) continue;
        for (int o = 0; o < 8; o++) {
            goff[l * 8 + o] = run;
            run += grp[l * 8 + o];
        }
    }
    const unsigned pool = run;
    int lv = 2;
    for (unsigned t = 0; t < pool; t += tile) {
        const unsigned cnt = min((unsigned)tile, pool - t), last = t + cnt - 1;
        // level of the tile's last cell: the pooled levels are in ascending order
        while (lv < depth) {
            const unsigned c = level_cells(lv);
            if (c <= (unsigned)pool_max && c > 0 && last < goff[lv * 8] + c) break;
            lv++;
        }
        M2LTile d;
        d.start = (int)t;
        d.count = (int)cnt;
        d.level = lv;
        d.octant = 8;
        tiles[nt++] = d;
    }
    for (int l = 2; l <= depth; l++) {
        if (level_cells(l) <= (unsigned)pool_max) continue;
        unsigned kmax = 0;
        for (int o = 0; o < 8; o++) {
            const unsigned c = grp[l * 8 + o];
            goff[l * 8 + o] = run;
            run += c;
            kmax = max(kmax, (c + tile - 1) / tile);
        }
        for (unsigned k = 0; k < kmax; k++)
            for (int o = 0; o < 8; o++) {
                const unsigned c = grp[l * 8 + o], t = k * tile;
                if (t >= c) continue;
                M2LTile d;
                d.start = (int)(goff[l * 8 + o] + t);
                d.count = (int)min((unsigned)tile, c - t);
                d.level = l;
                d.octant = o;
                tiles[nt++] = d;
            }
    }
    *ntiles = nt;
}

// A complete (level, octant) group (all 8^(l-1) cells present) is placed in
// the Morton order of its sub-lattice, so that every 128 consecutive entries
// are a block of 8 x 4 x 4 cells (x taking Morton bits 0, 3, 6, y 1, 4 and z
// 2, 5 of the halved position). With raster set (tiles of 128 rows) the
// entries inside each such block of a group of at least 512 cells are put in
// x, y, z order, row = x + 8 y + 32 z, the order in which the tensor-core M2L
// loads a shifted block of sources by TMA. Other groups in arrival order.
__global__ void oct_scatter_k(int c0, int nc, const int *__restrict__ level, const uint64_t *__restrict__ anchor,
                              const unsigned *__restrict__ grp, const unsigned *__restrict__ goff,
                              unsigned *__restrict__ fill, int raster, int *__restrict__ tgt)
{
    int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int l = level[c];
    const uint64_t code = anchor[c] >> (3 * (FMM_MAXLEVEL - l));
    int o = (int)(code & 7u);
    const bool complete = l <= 10 && grp[l * 8 + o] == (1u << (3 * (l - 1)));
    unsigned hm = (unsigned)(code >> 3);
    if (complete && raster && l >= 4) {
        const unsigned m = hm & 127u;
        const unsigned x = (m & 1u) | ((m >> 2) & 2u) | ((m >> 4) & 4u);
        const unsigned y = ((m >> 1) & 1u) | ((m >> 3) & 2u);
        const unsigned z = ((m >> 2) & 1u) | ((m >> 4) & 2u);
        hm = (hm & ~127u) | x | (y << 3) | (z << 5);
    }
    unsigned pos = goff[l * 8 + o] + (complete ? hm : atomicAdd(&fill[l * 8 + o], 1u));
    tgt[pos] = c;
}

__global__ void leaves_k(int nc, const int *__restrict__ nchild, unsigned *__restrict__ flag)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nc) flag[c] = nchild[c] == 0;
}

__global__ void leaves_write_k(int nc, const int *__restrict__ nchild, const unsigned *__restrict__ off,
                               int *__restrict__ leaves)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nc && nchild[c] == 0) leaves[off[c]] = c;
}

// leaf cell of every sorted particle: one warp per cell, leaves write their range
__global__ void pcell_k(int nc, const int *__restrict__ nchild, const int *__restrict__ begin,
                        const int *__restrict__ end, int *__restrict__ pcell)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (int)(t >> 5), lane = (int)(t & 31);
    if (c >= nc || nchild[c] != 0) return;
    for (int j = begin[c] + lane; j < end[c]; j += 32) pcell[j] = c;
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
// number of x in [0, S) of parity par with 0 <= x + v < S
static int64_t lattice_count(int64_t S, int par, int v)
{
    const int64_t lo = std::max<int64_t>(0, -v), hi = std::min<int64_t>(S, S - v);
    if (hi <= lo) return 0;
    return (hi + 1 - par) / 2 - (lo + 1 - par) / 2;
}

// Fast path of a full octree of depth L: P2P rows from the near-field stencil,
// no pairs across levels, and the implicit same-level M2L pairs counted in
// closed form (per level, octant and stencil vector, the cells of that octant
// whose partner lies inside the lattice). Returns false (nothing done) when
// the near stencil is longer than the row sort handles.
static bool uniform_lists(fmm_ctx *h, long long K0, cudaStream_t s)
{
    const int L = h->depth, nc = h->ncells;
    const int ls = h->lvl_start[L], le = h->lvl_start[L + 1];
    const double c = h->cmac;
    // offsets beyond the lattice side never land inside it
    const int R = (int)std::min<long long>((long long)std::ceil(std::sqrt((double)K0)) + 1, (1LL << L) - 1);
    std::vector<int> nv;
    for (int vx = -R; vx <= R; vx++)
        for (int vy = -R; vy <= R; vy++)
            for (int vz = -R; vz <= R; vz++) {
                const double d2 = (double)vx * vx + (double)vy * vy + (double)vz * vz;
                if (3.0 < c * d2) continue;
                if ((int)(nv.size() / 4) == ROW_SORT_CAP) return false;  // rows too long for the row sort
                nv.insert(nv.end(), {vx, vy, vz, 0});
            }
    const int nn = (int)(nv.size() / 4);
    h->near_dev.ensure(sizeof(int) * nv.size());
    FMM_CUDA_TRY(cudaMemcpyAsync(h->near_dev.p, nv.data(), sizeof(int) * nv.size(), cudaMemcpyHostToDevice, s));
    h->p2p_ptr.ensure(sizeof(int) * (size_t)(nc + 1));
    h->row_cnt.ensure(sizeof(unsigned) * (size_t)(nc + 1));
    FMM_CUDA_TRY(cudaMemsetAsync(h->row_cnt.p, 0, sizeof(unsigned) * (size_t)(nc + 1), s));
    near_rows_k<<<nblocks(le - ls, 128), 128, 0, s>>>(ls, le, L, h->c_xyz.as<int4>(), h->near_dev.as<int4>(), nn,
                                                      h->row_cnt.as<unsigned>(), nullptr, nullptr, false);
    count_launch(h);
    scan_exclusive_u32(h, h->row_cnt.as<unsigned>(), reinterpret_cast<unsigned *>(h->p2p_ptr.as<int>()), nc + 1, nullptr, s);
    unsigned *hp = h->hpin.as<unsigned>();
    FMM_CUDA_TRY(cudaMemcpyAsync(hp, h->p2p_ptr.as<int>() + nc, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    h->n_p2p = (int64_t)*hp;
    h->p2p_src.ensure(sizeof(int) * (size_t)std::max<int64_t>(h->n_p2p, 1));
    near_rows_k<<<nblocks(le - ls, 128), 128, 0, s>>>(ls, le, L, h->c_xyz.as<int4>(), h->near_dev.as<int4>(), nn,
                                                      nullptr, h->p2p_ptr.as<int>(), h->p2p_src.as<int>(), true);
    count_launch(h);
    row_sort_k<<<nblocks(nc, ROW_SORT_WARPS), 32 * ROW_SORT_WARPS, 0, s>>>(nc, h->p2p_ptr.as<int>(), h->p2p_src.as<int>());
    count_launch(h);
    check_launch("uniform lists");
    int64_t m2l = 0;
    for (int l = 1; l <= L; l++)
        for (int o = 0; o < 8; o++)
            for (int e = h->st_off[o]; e < h->st_off[o + 1]; e++) {
                const int *v = &h->st_host[4 * (size_t)e];
                m2l += lattice_count(1LL << l, o & 1, v[0]) * lattice_count(1LL << l, (o >> 1) & 1, v[1]) *
                       lattice_count(1LL << l, (o >> 2) & 1, v[2]);
            }
    h->n_m2l_implicit = m2l;
    h->n_m2lx = 0;
    return true;
}

void tree_build(fmm_ctx *h, const void *x, const void *q, int64_t n, int dt)
{
    cudaStream_t s = h->stream;
    const int TB = 256;
    h->box.ensure(sizeof(Box));
    Box *box = h->box.as<Box>();
    h->counters.ensure(sizeof(TravCounters) + 64 + sizeof(int) * 6 * (FMM_MAXLEVEL + 1));
    h->hpin.ensure(8192);

    // 1. bounding cube, keys
    box_init_k<<<1, 1, 0, s>>>(box);
    count_launch(h);
    const int bb_blocks = std::max(1, std::min((int)nblocks(n, TB), h->nsm * 8));
    if (dt == FMM_F64) bbox_k<double><<<bb_blocks, TB, 0, s>>>((const double *)x, n, box);
    else bbox_k<float><<<bb_blocks, TB, 0, s>>>((const float *)x, n, box);
    count_launch(h);
    box_final_k<<<1, 1, 0, s>>>(box);
    count_launch(h);
    h->keys.ensure(sizeof(uint64_t) * n);
    h->keys2.ensure(sizeof(uint64_t) * n);
    h->idx.ensure(sizeof(int) * n);
    h->idx2.ensure(sizeof(int) * n);
    if (dt == FMM_F64)
        keys_k<double><<<nblocks(n, TB), TB, 0, s>>>((const double *)x, n, box, h->keys.as<uint64_t>(), h->idx.as<int>());
    else
        keys_k<float><<<nblocks(n, TB), TB, 0, s>>>((const float *)x, n, box, h->keys.as<uint64_t>(), h->idx.as<int>());
    count_launch(h);
    check_launch("keys");

    // 2. sort
    if (radix_sort(h, h->keys.as<uint64_t>(), h->idx.as<int>(), h->keys2.as<uint64_t>(), h->idx2.as<int>(), n, 63, s)) {
        std::swap(h->keys, h->keys2);
        std::swap(h->idx, h->idx2);
    }

    // 3. sorted particles
    const bool mixed = h->precision == FMM_MIXED;
    const bool need64 = !mixed || dt == FMM_F64;
    if (need64) h->xs64.ensure(sizeof(double4_32a) * n);
    if (mixed) h->xs32.ensure(sizeof(float4) * n);
    double4_32a *xs64 = need64 ? h->xs64.as<double4_32a>() : nullptr;
    float4 *xs32 = mixed ? h->xs32.as<float4>() : nullptr;
    float4 *xs32lo = nullptr;
    if (mixed && dt == FMM_F64) {
        h->xs32lo.ensure(sizeof(float4) * n);
        xs32lo = h->xs32lo.as<float4>();
    }
    h->inv.ensure(sizeof(int) * n);
    if (dt == FMM_F64)
        gather_k<double><<<nblocks(n, TB), TB, 0, s>>>((const double *)x, (const double *)q, h->idx.as<int>(), n, xs64, xs32,
                                                       xs32lo, h->inv.as<int>());
    else
        gather_k<float><<<nblocks(n, TB), TB, 0, s>>>((const float *)x, (const float *)q, h->idx.as<int>(), n, xs64, xs32,
                                                      xs32lo, h->inv.as<int>());
    count_launch(h);
    check_launch("gather");

    // non-finite input is reported before any further work
    {
        int *hp = h->hpin.as<int>();
        FMM_CUDA_TRY(cudaMemcpyAsync(hp, &box->nonfinite, sizeof(int), cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        if (*hp) throw Error{FMM_ENONFINITE, "fmm_build: a position is NaN or infinite"};
    }

    // 4. cells, level by level
    // all cell arrays grow together; c_level's capacity stands for all of them
    auto grow_cells = [&](int need, int used) {
        size_t have = h->c_level.cap / sizeof(int);
        if (have >= (size_t)need) return;
        size_t want = std::max<size_t>((size_t)need, std::min<size_t>(2 * have, 0x7fffffff));
        h->c_level.ensure_keep(sizeof(int) * want, sizeof(int) * used, s);
        h->c_anchor.ensure_keep(sizeof(uint64_t) * want, sizeof(uint64_t) * used, s);
        h->c_begin.ensure_keep(sizeof(int) * want, sizeof(int) * used, s);
        h->c_end.ensure_keep(sizeof(int) * want, sizeof(int) * used, s);
        h->c_child.ensure_keep(sizeof(int) * want, sizeof(int) * used, s);
        h->c_nchild.ensure_keep(sizeof(int) * want, sizeof(int) * used, s);
        h->c_parent.ensure_keep(sizeof(int) * want, sizeof(int) * used, s);
        h->c_xyz.ensure_keep(sizeof(int4) * want, sizeof(int4) * used, s);
    };
    const int cap = (int)std::min<int64_t>(std::max<int64_t>(1024, 2 * (n / std::max(1, h->ncrit)) + 64), 0x7fffffff);
    grow_cells(cap, 0);
    root_k<<<1, 1, 0, s>>>((int)n, h->c_level.as<int>(), h->c_anchor.as<uint64_t>(), h->c_begin.as<int>(),
                           h->c_end.as<int>(), h->c_child.as<int>(), h->c_nchild.as<int>(), h->c_parent.as<int>(),
                           h->c_xyz.as<int4>());
    count_launch(h);
    h->lvl_start.assign(1, 0);
    h->lvl_start.push_back(1);
    int ncells = 1, depth = 0;
    for (int l = 0; l < FMM_MAXLEVEL; l++) {
        const int ls = h->lvl_start[l], le = h->lvl_start[l + 1];
        const int m = le - ls;
        if (m == 0) break;
        h->split_cnt.ensure(sizeof(unsigned) * (m + 1));
        h->split_off.ensure(sizeof(unsigned) * (m + 1));
        h->split_bnd.ensure(sizeof(int) * 9 * (size_t)m);
        split_count_k<<<nblocks(m, TB), TB, 0, s>>>(ls, le, l, h->ncrit, h->keys.as<uint64_t>(), h->c_begin.as<int>(),
                                                    h->c_end.as<int>(), h->split_cnt.as<unsigned>(), h->split_bnd.as<int>());
        count_launch(h);
        unsigned *tot = reinterpret_cast<unsigned *>(h->counters.as<char>() + sizeof(TravCounters));
        scan_exclusive_u32(h, h->split_cnt.as<unsigned>(), h->split_off.as<unsigned>(), m, tot, s);
        unsigned *hp = h->hpin.as<unsigned>();
        FMM_CUDA_TRY(cudaMemcpyAsync(hp, tot, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        const int nnew = (int)*hp;
        if ((int64_t)le + nnew > 0x7fffffffLL) throw Error{FMM_ENOMEM, "fmm_build: too many cells"};
        grow_cells(le + nnew, le);
        split_write_k<<<nblocks(m, TB), TB, 0, s>>>(ls, le, l, h->split_cnt.as<unsigned>(), h->split_off.as<unsigned>(),
                                                    h->split_bnd.as<int>(), h->c_level.as<int>(), h->c_anchor.as<uint64_t>(),
                                                    h->c_begin.as<int>(), h->c_end.as<int>(), h->c_child.as<int>(),
                                                    h->c_nchild.as<int>(), h->c_parent.as<int>(), h->c_xyz.as<int4>());
        count_launch(h);
        check_launch("cells");
        if (nnew == 0) break;
        h->lvl_start.push_back(le + nnew);
        ncells = le + nnew;
        depth = l + 1;
    }
    h->ncells = ncells;
    h->depth = depth;
    while ((int)h->lvl_start.size() < depth + 2) h->lvl_start.push_back(ncells);
    h->lvl_start.resize(depth + 2);

    // leaves
    {
        h->leaves.ensure(sizeof(int) * ncells);
        h->split_cnt.ensure(sizeof(unsigned) * (ncells + 1));
        h->split_off.ensure(sizeof(unsigned) * (ncells + 1));
        leaves_k<<<nblocks(ncells, TB), TB, 0, s>>>(ncells, h->c_nchild.as<int>(), h->split_cnt.as<unsigned>());
        count_launch(h);
        unsigned *tot = reinterpret_cast<unsigned *>(h->counters.as<char>() + sizeof(TravCounters));
        scan_exclusive_u32(h, h->split_cnt.as<unsigned>(), h->split_off.as<unsigned>(), ncells, tot, s);
        leaves_write_k<<<nblocks(ncells, TB), TB, 0, s>>>(ncells, h->c_nchild.as<int>(), h->split_off.as<unsigned>(),
                                                          h->leaves.as<int>());
        count_launch(h);
        h->pcell.ensure(sizeof(int) * (size_t)std::max<int64_t>(n, 1));
        pcell_k<<<nblocks((int64_t)ncells * 32, TB), TB, 0, s>>>(ncells, h->c_nchild.as<int>(), h->c_begin.as<int>(),
                                                               h->c_end.as<int>(), h->pcell.as<int>());
        count_launch(h);
        // lattice extent of the cells of every level: no same-level pair is
        // farther apart, which bounds the M2L stencil on deep adaptive trees
        constexpr int NE = 3 * (FMM_MAXLEVEL + 1);
        int *ext = reinterpret_cast<int *>(h->counters.as<char>() + sizeof(TravCounters) + 64);
        FMM_CUDA_TRY(cudaMemsetAsync(ext, 0x7f, sizeof(int) * NE, s));
        FMM_CUDA_TRY(cudaMemsetAsync(ext + NE, 0xff, sizeof(int) * NE, s));
        extent_k<<<nblocks(ncells, TB), TB, 0, s>>>(ncells, h->c_xyz.as<int4>(), ext);
        count_launch(h);
        unsigned *hp = h->hpin.as<unsigned>();
        int *hext = reinterpret_cast<int *>(h->hpin.as<char>() + 4096);
        FMM_CUDA_TRY(cudaMemcpyAsync(hp, tot, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaMemcpyAsync(hext, ext, sizeof(int) * 2 * NE, cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        h->nleaves = (int)*hp;
        int E = 0;
        h->lvl_ext.assign(FMM_MAXLEVEL + 1, -1);
        for (int l = 0; l <= depth; l++)
            for (int d = 0; d < 3; d++)
                if (hext[NE + 3 * l + d] >= hext[3 * l + d])
                    h->lvl_ext[l] = std::max(h->lvl_ext[l], hext[NE + 3 * l + d] - hext[3 * l + d]);
        for (int l = 0; l <= depth; l++) E = std::max(E, h->lvl_ext[l]);
        h->lattice_extent = E;
    }

    // 5. dual traversal
    stencil_update(h);
    stencil_levels(h, s);
    long long K0 = (long long)std::ceil(3.0 / h->cmac);
    while (K0 > 0 && 3.0 < h->cmac * (double)(K0 - 1)) K0--;
    while (!(3.0 < h->cmac * (double)K0)) K0++;
    // a full octree (all leaves on the deepest level, every level full) takes
    // the lattice stencils instead of the traversal
    bool full = h->uniform_req && depth >= 1 && depth <= 9 && h->nleaves == (1 << (3 * depth)) &&
                (int64_t)ncells == (((int64_t)1 << (3 * (depth + 1))) - 1) / 7;
    if (full) full = uniform_lists(h, K0, s);
    h->uniform_used = full;
    if (!full) {
        // the near-field stencil size bounds the P2P list of a leaf in a uniform tree
        const size_t per = (size_t)h->p2p_cap_hint + 8;
        size_t cap_p2p = std::max<size_t>(1024, std::min((size_t)h->nleaves * per, (size_t)h->nleaves * h->nleaves));
        size_t cap_m2lx = std::max<size_t>(1024, (size_t)ncells * 4);
        size_t cap_next = std::max<size_t>(1024, std::min((size_t)ncells * per, (size_t)ncells * ncells));
        h->p2p_pairs.ensure(sizeof(int2) * cap_p2p);
        h->m2lx_pairs.ensure(sizeof(int2) * cap_m2lx);
        h->frontA.ensure(sizeof(int2) * cap_next);
        h->frontB.ensure(sizeof(int2) * cap_next);
        cap_p2p = h->p2p_pairs.cap / sizeof(int2);
        cap_m2lx = h->m2lx_pairs.cap / sizeof(int2);
        TravCounters *dc = h->counters.as<TravCounters>();
        TravCounters hc = {0, 0, 0, 0};
        TravCounters *hp = h->hpin.as<TravCounters>();
        int64_t nF = 0;
        if (ncells == 1) {
            // the root is a leaf: one self pair
            int2 rp = make_int2(0, 0);
            FMM_CUDA_TRY(cudaMemcpyAsync(h->p2p_pairs.p, &rp, sizeof(int2), cudaMemcpyHostToDevice, s));
            FMM_CUDA_TRY(cudaStreamSynchronize(s));
            hc.n_p2p = 1;
        } else {
            int2 rp = make_int2(0, 0);
            FMM_CUDA_TRY(cudaMemcpyAsync(h->frontA.p, &rp, sizeof(int2), cudaMemcpyHostToDevice, s));
            FMM_CUDA_TRY(cudaStreamSynchronize(s));
            nF = 1;
        }
        while (nF > 0) {
            if (nF > 0x7fffffffLL) throw Error{FMM_ENOMEM, "fmm_build: traversal frontier too large"};
            for (int attempt = 0; attempt < 8; attempt++) {
                TravCounters start = hc;
                start.n_next = 0;
                *hp = start;
                FMM_CUDA_TRY(cudaMemcpyAsync(dc, hp, sizeof(TravCounters), cudaMemcpyHostToDevice, s));
                size_t cn = h->frontB.cap / sizeof(int2);
                expand_k<<<nblocks(nF * 8, 256), 256, 0, s>>>(h->frontA.as<int2>(), (unsigned)nF, h->c_xyz.as<int4>(),
                                                          h->c_child.as<int>(), h->c_nchild.as<int>(), h->cmac, K0,
                                                          h->p2p_pairs.as<int2>(), cap_p2p, h->m2lx_pairs.as<int2>(),
                                                          cap_m2lx, h->frontB.as<int2>(), cn, dc);
                count_launch(h);
                check_launch("traversal");
                FMM_CUDA_TRY(cudaMemcpyAsync(hp, dc, sizeof(TravCounters), cudaMemcpyDeviceToHost, s));
                FMM_CUDA_TRY(cudaStreamSynchronize(s));
                TravCounters got = *hp;
                bool over = false;
                if (got.n_p2p > cap_p2p) {
                    h->p2p_pairs.ensure_keep(sizeof(int2) * (size_t)(got.n_p2p * 5 / 4 + 1024), sizeof(int2) * start.n_p2p, s);
                    cap_p2p = h->p2p_pairs.cap / sizeof(int2);
                    over = true;
                }
                if (got.n_m2lx > cap_m2lx) {
                    h->m2lx_pairs.ensure_keep(sizeof(int2) * (size_t)(got.n_m2lx * 5 / 4 + 1024), sizeof(int2) * start.n_m2lx, s);
                    cap_m2lx = h->m2lx_pairs.cap / sizeof(int2);
                    over = true;
                }
                if (got.n_next > cn) {
                    h->frontB.ensure(sizeof(int2) * (size_t)(got.n_next * 5 / 4 + 1024));
                    over = true;
                }
                if (!over) {
                    hc = got;
                    break;
                }
                if (attempt == 7) throw Error{FMM_ENOMEM, "fmm_build: traversal buffers keep overflowing"};
            }
            nF = (int64_t)hc.n_next;
            std::swap(h->frontA, h->frontB);
            if (h->frontB.cap < h->frontA.cap) h->frontB.ensure(h->frontA.cap);
        }
        h->n_p2p = (int64_t)hc.n_p2p;
        h->n_m2lx = (int64_t)hc.n_m2lx;
        h->n_m2l_implicit = (int64_t)hc.n_m2l_implicit;
        if (h->n_p2p > 0x7fffffffLL || h->n_m2lx > 0x7fffffffLL)
            throw Error{FMM_ENOMEM, "fmm_build: interaction lists exceed 2^31 entries"};
        h->p2p_cap_hint = (int)std::max<int64_t>(h->p2p_cap_hint, h->n_p2p / std::max(1, h->nleaves) + 1);
    }

    // 6. CSR lists
    if (!full) pairs_to_csr(h, h->p2p_pairs.as<int2>(), h->n_p2p, h->p2p_ptr, h->p2p_src, s);
    pairs_to_csr(h, h->m2lx_pairs.as<int2>(), h->n_m2lx, h->m2lx_ptr, h->m2lx_src, s);
    h->p2p_runs.ensure(sizeof(int2) * (size_t)std::max<int64_t>(h->n_p2p, 1));
    h->p2p_nrun.ensure(sizeof(int) * (size_t)ncells);
    if (h->nleaves > 0) {
        p2p_runs_k<<<nblocks(h->nleaves, 128), 128, 0, s>>>(h->nleaves, h->leaves.as<int>(), h->p2p_ptr.as<int>(),
                                                            h->p2p_src.as<int>(), h->c_begin.as<int>(), h->c_end.as<int>(),
                                                            h->p2p_runs.as<int2>(), h->p2p_nrun.as<int>());
        count_launch(h);
        check_launch("p2p runs");
    }
    p2p_prepare(h, s);
    {
        unsigned long long *acc = reinterpret_cast<unsigned long long *>(h->counters.as<char>() + sizeof(TravCounters) + 8);
        FMM_CUDA_TRY(cudaMemsetAsync(acc, 0, 8, s));
        interactions_k<<<nblocks(ncells, 256), 256, 0, s>>>(h->p2p_ptr.as<int>(), h->p2p_src.as<int>(), h->c_begin.as<int>(),
                                                            h->c_end.as<int>(), ncells, acc);
        count_launch(h);
        unsigned long long *hp = h->hpin.as<unsigned long long>();
        FMM_CUDA_TRY(cudaMemcpyAsync(hp, acc, 8, cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        h->n_interactions = (int64_t)*hp - n;
    }

    // 7. per-level lattice maps
    {
        std::vector<LevelDesc> ld(FMM_MAXLEVEL + 1);
        long long pool = 0;
        for (int l = 0; l <= FMM_MAXLEVEL; l++) {
            ld[l].start = l <= depth ? h->lvl_start[l] : ncells;
            ld[l].end = l <= depth ? h->lvl_start[l + 1] : ncells;
            ld[l].map_off = -1;
            if (l >= 2 && l <= depth && l <= FMM_DENSE_MAP_MAXLEVEL) {
                ld[l].map_off = pool;
                pool += 1LL << (3 * l);
            }
        }
        h->map_pool.ensure(sizeof(int) * (size_t)std::max<long long>(pool, 1));
        if (pool > 0) FMM_CUDA_TRY(cudaMemsetAsync(h->map_pool.p, 0xff, sizeof(int) * (size_t)pool, s));
        for (int l = 2; l <= depth && l <= FMM_DENSE_MAP_MAXLEVEL; l++) {
            int m = ld[l].end - ld[l].start;
            if (m == 0) continue;
            map_fill_k<<<nblocks(m, TB), TB, 0, s>>>(ld[l].start, ld[l].end, l, h->c_anchor.as<uint64_t>(),
                                                     h->map_pool.as<int>() + ld[l].map_off);
            count_launch(h);
        }
        // deeper levels: hash tables of at least twice their cells
        std::vector<long long> hoff(FMM_MAXLEVEL + 1, -1);
        long long hpool = 0;
        for (int l = FMM_DENSE_MAP_MAXLEVEL + 1; l <= depth; l++) {
            const long long m = ld[l].end - ld[l].start;
            ld[l].hash = nullptr;
            ld[l].hash_mask = 0;
            if (m == 0) continue;
            long long t = 64;
            while (t < 2 * m) t <<= 1;
            hoff[l] = hpool;
            ld[l].hash_mask = (unsigned)(t - 1);
            hpool += t;
        }
        if (hpool > 0) {
            h->hash_pool.ensure(sizeof(HashSlot) * (size_t)hpool);
            FMM_CUDA_TRY(cudaMemsetAsync(h->hash_pool.p, 0, sizeof(HashSlot) * (size_t)hpool, s));
            for (int l = FMM_DENSE_MAP_MAXLEVEL + 1; l <= depth; l++) {
                if (hoff[l] < 0) continue;
                HashSlot *tab = h->hash_pool.as<HashSlot>() + hoff[l];
                ld[l].hash = tab;
                const int m = ld[l].end - ld[l].start;
                hash_fill_k<<<nblocks(m, TB), TB, 0, s>>>(ld[l].start, ld[l].end, l, h->c_anchor.as<uint64_t>(), tab,
                                                          ld[l].hash_mask);
                count_launch(h);
            }
        }
        h->lvl_desc.ensure(sizeof(LevelDesc) * ld.size());
        LevelDesc *hp = reinterpret_cast<LevelDesc *>(h->hpin.as<char>() + 1024);
        std::copy(ld.begin(), ld.end(), hp);
        FMM_CUDA_TRY(cudaMemcpyAsync(h->lvl_desc.p, hp, sizeof(LevelDesc) * ld.size(), cudaMemcpyHostToDevice, s));
        check_launch("maps");
    }

    // 8. M2L target tiles: cells of levels >= 2 grouped by (level, octant)
    {
        const int tile = m2l_tile_size(h);
        const int c0 = depth >= 2 ? h->lvl_start[2] : ncells;
        const int nt = ncells - c0;
        h->ntiles_max = nt / tile + 8 * (FMM_MAXLEVEL + 1) + 1;
        h->m2l_tgt.ensure(sizeof(int) * (size_t)std::max(nt, 1));
        h->m2l_tiles.ensure(sizeof(M2LTile) * (size_t)h->ntiles_max);
        h->m2l_misc.ensure(sizeof(unsigned) * 3 * 8 * (FMM_MAXLEVEL + 1) + 64);
        unsigned *grp = h->m2l_misc.as<unsigned>();
        unsigned *goff = grp + 8 * (FMM_MAXLEVEL + 1);
        unsigned *fill = goff + 8 * (FMM_MAXLEVEL + 1);
        int *ntiles = reinterpret_cast<int *>(fill + 8 * (FMM_MAXLEVEL + 1));
        FMM_CUDA_TRY(cudaMemsetAsync(grp, 0, sizeof(unsigned) * 3 * 8 * (FMM_MAXLEVEL + 1) + 64, s));
        if (nt > 0) {
            oct_count_k<<<nblocks(nt, TB), TB, 0, s>>>(c0, ncells, h->c_level.as<int>(), h->c_anchor.as<uint64_t>(), grp);
            count_launch(h);
        }
        const int pool_max = h->m2l_pool >= 0 ? h->m2l_pool : 4 * tile;
        tiles_k<<<1, 1, 0, s>>>(depth, tile, pool_max, grp, goff, h->m2l_tiles.as<M2LTile>(), ntiles);
        count_launch(h);
        if (nt > 0) {
            oct_scatter_k<<<nblocks(nt, TB), TB, 0, s>>>(c0, ncells, h->c_level.as<int>(), h->c_anchor.as<uint64_t>(),
                                                         grp, goff, fill, tile == 128 ? 1 : 0, h->m2l_tgt.as<int>());
            count_launch(h);
        }
        check_launch("m2l tiles");
        lattice_prepare(h, s);
    }
}

int64_t tree_m2l_total(fmm_ctx *h) { return h->n_m2l_implicit + h->n_m2lx; }

// ---------------------------------------------------------------------------
// export (tests): the implicit same-level M2L pairs are enumerated from the
// stencil and merged with the explicit ones
// ---------------------------------------------------------------------------
__global__ void stencil_pairs_k(int c0, int nc, const int *__restrict__ level, const int4 *__restrict__ xyz,
                                const uint64_t *__restrict__ anchor, const LevelDesc *__restrict__ ld,
                                const int *__restrict__ map_pool, const int4 *__restrict__ st, const int *__restrict__ st_off,
                                unsigned *__restrict__ cnt, const unsigned *__restrict__ off, int2 *__restrict__ out)
{
    int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int l = level[c];
    const int4 a = xyz[c];
    const int sh = FMM_MAXLEVEL - l;
    const int px = a.x >> sh, py = a.y >> sh, pz = a.z >> sh;
    const int o = (px & 1) | ((py & 1) << 1) | ((pz & 1) << 2);
    const LevelDesc L = ld[l];
    unsigned k = 0;
    unsigned base = off ? off[c - c0] : 0;
    for (int e = st_off[o]; e < st_off[o + 1]; e++) {
        int4 v = st[e];
        int b = level_lookup(L, map_pool, anchor, l, px + v.x, py + v.y, pz + v.z);
        if (b < 0) continue;
        if (out) out[base + k] = make_int2(c, b);
        k++;
    }
    if (!out) cnt[c - c0] = k;
}

void tree_export(fmm_ctx *h, uint64_t *keys, int32_t *perm, int32_t *level, uint64_t *anchor, int32_t *begin,
                 int32_t *end, int32_t *child, int32_t *nchild, int32_t *parent, int64_t *p2p_ptr, int32_t *p2p_idx,
                 int64_t *m2l_ptr, int32_t *m2l_idx, double *box)
{
    cudaStream_t s = h->stream;
    const int nc = h->ncells;
    const int64_t n = h->n;
    auto d2h = [&](void *dst, const void *src, size_t bytes) {
        if (dst && bytes) FMM_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
    };
    d2h(keys, h->keys.p, sizeof(uint64_t) * n);
    d2h(perm, h->idx.p, sizeof(int) * n);
    d2h(level, h->c_level.p, sizeof(int) * nc);
    d2h(anchor, h->c_anchor.p, sizeof(uint64_t) * nc);
    d2h(begin, h->c_begin.p, sizeof(int) * nc);
    d2h(end, h->c_end.p, sizeof(int) * nc);
    d2h(child, h->c_child.p, sizeof(int) * nc);
    d2h(nchild, h->c_nchild.p, sizeof(int) * nc);
    d2h(parent, h->c_parent.p, sizeof(int) * nc);
    if (box) {
        Box hb;
        FMM_CUDA_TRY(cudaMemcpyAsync(&hb, h->box.p, sizeof(Box), cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        box[0] = hb.origin[0];
        box[1] = hb.origin[1];
        box[2] = hb.origin[2];
        box[3] = hb.R0;
    }
    if (p2p_ptr || p2p_idx) {
        std::vector<int> ptr(nc + 1);
        FMM_CUDA_TRY(cudaMemcpyAsync(ptr.data(), h->p2p_ptr.p, sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost, s));
        d2h(p2p_idx, h->p2p_src.p, sizeof(int) * h->n_p2p);
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        if (p2p_ptr)
            for (int i = 0; i <= nc; i++) p2p_ptr[i] = ptr[i];
    }
    if (m2l_ptr || m2l_idx) {
        // implicit same-level pairs: count, scan, write
        const int c0 = h->depth >= 2 ? h->lvl_start[2] : nc;
        const int m = nc - c0;
        int64_t nimp = 0;
        DevBuf cnt, off, pairs, ptr, src;
        if (m > 0) {
            cnt.ensure(sizeof(unsigned) * (m + 1));
            off.ensure(sizeof(unsigned) * (m + 1));
            const int *st_off = stencil_offsets(h);
            stencil_pairs_k<<<nblocks(m, 128), 128, 0, s>>>(c0, nc, h->c_level.as<int>(), h->c_xyz.as<int4>(),
                                                            h->c_anchor.as<uint64_t>(), h->lvl_desc.as<LevelDesc>(),
                                                            h->map_pool.as<int>(), h->st_dev.as<int4>(), st_off,
                                                            cnt.as<unsigned>(), nullptr, nullptr);
            count_launch(h);
            unsigned *tot = reinterpret_cast<unsigned *>(h->counters.as<char>() + sizeof(TravCounters));
            scan_exclusive_u32(h, cnt.as<unsigned>(), off.as<unsigned>(), m, tot, s);
            unsigned ht = 0;
            FMM_CUDA_TRY(cudaMemcpyAsync(&ht, tot, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
            FMM_CUDA_TRY(cudaStreamSynchronize(s));
            nimp = ht;
        }
        const int64_t ntot = nimp + h->n_m2lx;
        pairs.ensure(sizeof(int2) * (size_t)std::max<int64_t>(ntot, 1));
        if (m > 0 && nimp > 0) {
            const int *st_off = stencil_offsets(h);
            stencil_pairs_k<<<nblocks(m, 128), 128, 0, s>>>(c0, nc, h->c_level.as<int>(), h->c_xyz.as<int4>(),
                                                            h->c_anchor.as<uint64_t>(), h->lvl_desc.as<LevelDesc>(),
                                                            h->map_pool.as<int>(), h->st_dev.as<int4>(), st_off,
                                                            cnt.as<unsigned>(), off.as<unsigned>(), pairs.as<int2>());
            count_launch(h);
        }
        if (h->n_m2lx > 0)
            FMM_CUDA_TRY(cudaMemcpyAsync(pairs.as<int2>() + nimp, h->m2lx_pairs.p, sizeof(int2) * h->n_m2lx,
                                         cudaMemcpyDeviceToDevice, s));
        pairs_to_csr(h, pairs.as<int2>(), ntot, ptr, src, s);
        std::vector<int> hptr(nc + 1);
        FMM_CUDA_TRY(cudaMemcpyAsync(hptr.data(), ptr.p, sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost, s));
        d2h(m2l_idx, src.p, sizeof(int) * ntot);
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        if (m2l_ptr)
            for (int i = 0; i <= nc; i++) m2l_ptr[i] = hptr[i];
        cnt.release();
        off.release();
        pairs.release();
        ptr.release();
        src.release();
    }
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
}

}  // namespace fmm
