// Multipole and local expansions: P2M, M2M, M2L, L2L and L2P (Sec. 2.1 and
// Fig. flow_chart of Yokota & Barba, arXiv:1106.2176), over solid harmonics of
// p terms (degrees 0..p-1).
//
// Basis: R_n^m(x) = r^n P_n^m(cos t) e^{imf} / (n+m)!  and
//        I_n^m(x) = (n-m)! P_n^m(cos t) e^{imf} / r^(n+1),
// P_n^m without the Condon-Shortley phase, X_n^{-m} = (-1)^m conj(X_n^m). They
// are generated here from Cartesian three-term recurrences (no trigonometry):
//   R_m^m = R_{m-1}^{m-1} (x + iy) / (2m),   R_{m+1}^m = z R_m^m,
//   (n+m)(n-m) R_n^m = (2n-1) z R_{n-1}^m - r^2 R_{n-2}^m;
//   I_0^0 = 1/r,  I_m^m = (2m-1) (x + iy) / r^2 I_{m-1}^{m-1},
//   I_{m+1}^m = (2m+1) z / r^2 I_m^m,
//   r^2 I_n^m = (2n-1) z I_{n-1}^m - (n+m-1)(n-m-1) I_{n-2}^m.
//
// Every expansion is stored scaled by the width w of its cell, M_n^m / w^n and
// L_n^m w^(n+1); then the same-level M2L operator depends only on the integer
// lattice offset of the two cells and M2M / L2L only on the child octant:
//   M2M  M~p(n,m) = sum_{k,l} conj(R_k^l(t)) M~c(n-k, m-l) 2^-(n-k),  t = (c_c - c_p)/w_p
//   M2L  L~A(n,m) += (-1)^n sum_{j,k} M~B(j,k) I_{j+n}^{k+m}(u),      u = (c_A - c_B)/w
//   L2L  L~c(k,l) += 2^-(k+1) sum_{n,m} L~p(n,m) conj(R_{n-k}^{m-l}(t))
//   P2M  M~(n,m)  = sum_j q_j conj(R_n^m((x_j - c)/w))
//   L2P  phi = Re sum L~ conj(R(x^)) / w, grad from d_z R_n^m = R_{n-1}^m and
//        (d_x + i d_y) R_n^m = -R_{n-1}^{m+1}, divided by w^2.
#include <algorithm>
#include <climits>
#include <array>
#include <type_traits>
#include <cmath>
#include <map>
#include <tuple>

#include "fmm_internal.cuh"
#include "m2lx_layout.cuh"

namespace fmm {

static inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__host__ __device__ inline int tri(int n, int m) { return n * (n + 1) / 2 + m; }
__host__ __device__ inline int full(int n, int m) { return n * n + n + m; }

// R_n^m, 0 <= m <= n < P, triangular storage, element k at re[k * st]
template <class T>
__host__ __device__ void regular_tri(int P, T x, T y, T z, T *re, T *im, int st)
{
    const T r2 = x * x + y * y + z * z;
    T mre = T(1), mim = T(0);
    for (int m = 0; m < P; m++) {
        if (m > 0) {
            const T f = T(1) / T(2 * m);
            const T a = (mre * x - mim * y) * f;
            const T b = (mre * y + mim * x) * f;
            mre = a;
            mim = b;
        }
        re[tri(m, m) * st] = mre;
        im[tri(m, m) * st] = mim;
        if (m + 1 >= P) continue;
        T p2re = mre, p2im = mim, p1re = z * mre, p1im = z * mim;
        re[tri(m + 1, m) * st] = p1re;
        im[tri(m + 1, m) * st] = p1im;
        for (int n = m + 2; n < P; n++) {
            const T a = T(2 * n - 1), b = T(1) / T((n + m) * (n - m));
            const T cre = (a * z * p1re - r2 * p2re) * b;
            const T cim = (a * z * p1im - r2 * p2im) * b;
            re[tri(n, m) * st] = cre;
            im[tri(n, m) * st] = cim;
            p2re = p1re; p2im = p1im; p1re = cre; p1im = cim;
        }
    }
}

// complex coefficient (n, m), any -n <= m <= n, of a packed real expansion
template <class T>
__device__ __forceinline__ void cget(const T *__restrict__ X, int n, int m, T &re, T &im)
{
    const int a = m < 0 ? -m : m;
    re = X[re_idx(n, a)];
    im = a ? X[im_idx(n, a)] : T(0);
    if (m < 0) {
        im = -im;
        if (a & 1) {
            re = -re;
            im = -im;
        }
    }
}

__device__ __forceinline__ void tri_inv(int k, int &n, int &m)
{
    n = (int)((sqrtf(8.0f * k + 1.0f) - 1.0f) * 0.5f);
    while (tri(n + 1, 0) <= k) n++;
    while (tri(n, 0) > k) n--;
    m = k - tri(n, 0);
}

// geometric centre and width of a cell: origin + (anchor + 2^(20-l)) h, w = h 2^(21-l)
__device__ __forceinline__ void cell_geom(const Box *__restrict__ b, int4 a, double c[3], double &w)
{
    const double h = b->h;
    const double half = ldexp(1.0, FMM_MAXLEVEL - 1 - a.w);
    c[0] = __dadd_rn(b->origin[0], __dmul_rn((double)a.x + half, h));
    c[1] = __dadd_rn(b->origin[1], __dmul_rn((double)a.y + half, h));
    c[2] = __dadd_rn(b->origin[2], __dmul_rn((double)a.z + half, h));
    w = ldexp(h, FMM_MAXLEVEL - a.w);
}

__device__ __forceinline__ int child_octant(int4 a)
{
    const int bit = FMM_MAXLEVEL - a.w;
    return ((a.x >> bit) & 1) | (((a.y >> bit) & 1) << 1) | (((a.z >> bit) & 1) << 2);
}

// particle j relative to the cell centre c, in FP64
__device__ __forceinline__ double4_32a rel_pt(const double4_32a *p, int j, const double c[3])
{
    const double4_32a v = p[j];
    return make_double4_32a(v.x - c[0], v.y - c[1], v.z - c[2], v.w);
}
__device__ __forceinline__ double4_32a rel_pt(const float4 *p, int j, const double c[3])
{
    const float4 v = p[j];
    return make_double4_32a((double)v.x - c[0], (double)v.y - c[1], (double)v.z - c[2], v.w);
}

// ---------------------------------------------------------------------------
// P2M: one block per leaf, a chunk of particles at a time
// ---------------------------------------------------------------------------
template <class T, class P4>
__global__ void __launch_bounds__(64) p2m_k(int p, const int *__restrict__ leaves, const int *__restrict__ begin,
                                            const int *__restrict__ end, const int4 *__restrict__ xyz,
                                            const Box *__restrict__ box, const P4 *__restrict__ xs, T *__restrict__ M,
                                            int chunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ntri = p * (p + 1) / 2, PP = p * p;
    T *sre = reinterpret_cast<T *>(smem_raw);
    T *sim = sre + chunk * ntri;
    const int c = leaves[blockIdx.x];
    double cen[3], w;
    cell_geom(box, xyz[c], cen, w);
    const double iw = 1.0 / w;
    const int b = begin[c], e = end[c];
    T are[4] = {0, 0, 0, 0}, aim[4] = {0, 0, 0, 0};
    for (int j0 = b; j0 < e; j0 += chunk) {
        const int t = threadIdx.x;
        if (t < chunk) {
            const int j = j0 + t;
            if (j < e) {
                const double4_32a pt = rel_pt(xs, j, cen);
                const T dx = (T)(pt.x * iw), dy = (T)(pt.y * iw), dz = (T)(pt.z * iw);
                regular_tri<T>(p, dx, dy, dz, sre + t, sim + t, chunk);
                const T q = (T)pt.w;
                for (int k = 0; k < ntri; k++) {
                    sre[k * chunk + t] *= q;
                    sim[k * chunk + t] *= -q;
                }
            } else {
                for (int k = 0; k < ntri; k++) {
                    sre[k * chunk + t] = T(0);
                    sim[k * chunk + t] = T(0);
                }
            }
        }
        __syncthreads();
        for (int r = 0; r < 4; r++) {
            const int k = threadIdx.x + r * blockDim.x;
            if (k >= ntri) break;
            T sr = 0, si = 0;
            for (int tt = 0; tt < chunk; tt++) {
                sr += sre[k * chunk + tt];
                si += sim[k * chunk + tt];
            }
            are[r] += sr;
            aim[r] += si;
        }
        __syncthreads();
    }
    T *Mc = M + (size_t)c * PP;
    for (int r = 0; r < 4; r++) {
        const int k = threadIdx.x + r * blockDim.x;
        if (k >= ntri) break;
        int n, m;
        tri_inv(k, n, m);
        Mc[re_idx(n, m)] = are[r];
        if (m) Mc[im_idx(n, m)] = aim[r];
    }
}

// P2M with the order fixed at compile time: one warp per leaf, each lane runs
// the regular-harmonic recurrences of its particles in registers and adds
// q conj(R_n^m) into its own accumulators; a butterfly over the warp sums them
// and lane k writes coefficients k, k+32, ...  (Sec. 2.1, P2M.)
template <int P, class T>
__device__ __forceinline__ void p2m_accum(T x, T y, T z, T q, T *are, T *aim)
{
    const T r2 = x * x + y * y + z * z;
    T mre = T(1), mim = T(0);
#pragma unroll
    for (int m = 0; m < P; m++) {
        if (m > 0) {
            const T f = T(1) / T(2 * m);
            const T a = (mre * x - mim * y) * f;
            const T b = (mre * y + mim * x) * f;
            mre = a;
            mim = b;
        }
        are[tri(m, m)] += q * mre;
        aim[tri(m, m)] -= q * mim;
        if (m + 1 < P) {
            T p2re = mre, p2im = mim, p1re = z * mre, p1im = z * mim;
            are[tri(m + 1, m)] += q * p1re;
            aim[tri(m + 1, m)] -= q * p1im;
#pragma unroll
            for (int n = m + 2; n < P; n++) {
                const T a = T(2 * n - 1), b = T(1) / T((n + m) * (n - m));
                const T cre = (a * z * p1re - r2 * p2re) * b;
                const T cim = (a * z * p1im - r2 * p2im) * b;
                are[tri(n, m)] += q * cre;
                aim[tri(n, m)] -= q * cim;
                p2re = p1re; p2im = p1im; p1re = cre; p1im = cim;
            }
        }
    }
}

constexpr int P2M_WARPS = 8;
constexpr int P2M_WARP_MAXP = 10;

// P2M of leaf c by one warp (lane = threadIdx.x & 31)
template <int P, class P4>
__device__ __forceinline__ void p2m_leaf_warp(int c, int lane, const int *__restrict__ begin, const int *__restrict__ end,
                                              const int4 *__restrict__ xyz, const Box *__restrict__ box,
                                              const P4 *__restrict__ xs, float *__restrict__ M)
{
    constexpr int NT = P * (P + 1) / 2;
    double cen[3], w;
    cell_geom(box, xyz[c], cen, w);
    const double iw = 1.0 / w;
    const int b = begin[c], e = end[c];
    float are[NT], aim[NT];
#pragma unroll
    for (int k = 0; k < NT; k++) are[k] = aim[k] = 0.f;
    for (int j = b + lane; j < e; j += 32) {
        const double4_32a pt = rel_pt(xs, j, cen);
        p2m_accum<P, float>((float)(pt.x * iw), (float)(pt.y * iw), (float)(pt.z * iw), (float)pt.w, are, aim);
    }
    // sum over the 32 lanes by recursive halving: the 2 NT values (padded to
    // VP, a multiple of 32) are split in two at every step, each lane keeping
    // the half its lane bit selects and adding its partner's copy of that
    // half, so that lane l ends with the sums of values [l W, (l + 1) W)
    constexpr int VP = (2 * NT + 31) / 32 * 32, W = VP / 32;
    float v[VP];
#pragma unroll
    for (int i = 0; i < VP; i++) v[i] = i < NT ? are[i] : (i < 2 * NT ? aim[i - NT] : 0.f);
#pragma unroll
    for (int o = 16, h = VP / 2; o; o >>= 1, h >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; i++) {
            const float keep = up ? v[i + h] : v[i], send = up ? v[i] : v[i + h];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    float *Mc = M + (size_t)c * (P * P);
#pragma unroll
    for (int t = 0; t < W; t++) {
        const int i = lane * W + t;
        if (i < 2 * NT) {
            const int k = i < NT ? i : i - NT;
            int n = 0;
            while ((n + 1) * (n + 2) / 2 <= k) n++;
            const int m = k - n * (n + 1) / 2;
            if (i < NT) Mc[re_idx(n, m)] = v[t];
            else if (m) Mc[im_idx(n, m)] = v[t];
        }
    }
}

template <int P, class P4>
__global__ void __launch_bounds__(32 * P2M_WARPS) p2m_warp_k(int nleaves, const int *__restrict__ leaves,
                                                             const int *__restrict__ begin, const int *__restrict__ end,
                                                             const int4 *__restrict__ xyz, const Box *__restrict__ box,
                                                             const P4 *__restrict__ xs, float *__restrict__ M)
{
    const int li = blockIdx.x * P2M_WARPS + (threadIdx.x >> 5);
    if (li >= nleaves) return;
    p2m_leaf_warp<P, P4>(leaves[li], threadIdx.x & 31, begin, end, xyz, box, xs, M);
}

template <class P4>
static bool p2m_warp_launch(int p, int nleaves, const int *leaves, const int *begin, const int *end, const int4 *xyz,
                            const Box *box, const P4 *xs, float *M, cudaStream_t s)
{
    const unsigned g = nblk(nleaves, P2M_WARPS);
    const unsigned bs = 32 * P2M_WARPS;
    switch (p) {
#define FMM_P2M_CASE(PV) \
    case PV: p2m_warp_k<PV, P4><<<g, bs, 0, s>>>(nleaves, leaves, begin, end, xyz, box, xs, M); return true;
        FMM_P2M_CASE(2) FMM_P2M_CASE(3) FMM_P2M_CASE(4) FMM_P2M_CASE(5) FMM_P2M_CASE(6)
        FMM_P2M_CASE(7) FMM_P2M_CASE(8) FMM_P2M_CASE(9) FMM_P2M_CASE(10)
#undef FMM_P2M_CASE
    default: return false;
    }
}
static_assert(P2M_WARP_MAXP == 10, "p2m_warp_launch instantiates p = 2 .. 10");

// ---------------------------------------------------------------------------
// M2M: one thread per (parent cell, output coefficient)
// ---------------------------------------------------------------------------
template <class T>
__global__ void m2m_k(int p, int ls, int le, const int *__restrict__ child, const int *__restrict__ nchild,
                      const int4 *__restrict__ xyz, const T *__restrict__ rtab, T *__restrict__ M)
{
    const int ntri = p * (p + 1) / 2, PP = p * p;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = ls + (int)(gid / ntri);
    const int ci = (int)(gid % ntri);
    if (c >= le) return;
    const int nc = nchild[c];
    if (nc == 0) return;
    int n, m;
    tri_inv(ci, n, m);
    T sr = 0, si = 0;
    const int c0 = child[c];
    for (int ch = c0; ch < c0 + nc; ch++) {
        const T *R = rtab + (size_t)child_octant(xyz[ch]) * PP * 2;
        const T *Mc = M + (size_t)ch * PP;
        for (int k = 0; k <= n; k++) {
            const int j = n - k;
            const T sc = (T)ldexp(1.0, -j);
            for (int l = -k; l <= k; l++) {
                const int mu = m - l;
                if (mu > j || mu < -j) continue;
                const T rr = R[2 * full(k, l)], ri = -R[2 * full(k, l) + 1];  // conj(R)
                T mr, mi;
                cget(Mc, j, mu, mr, mi);
                sr += sc * (rr * mr - ri * mi);
                si += sc * (rr * mi + ri * mr);
            }
        }
    }
    T *Mp = M + (size_t)c * PP;
    Mp[re_idx(n, m)] = sr;
    if (m) Mp[im_idx(n, m)] = si;
}

// ---------------------------------------------------------------------------
// L2L: one thread per (child cell, output coefficient), parent level done
// ---------------------------------------------------------------------------
template <class T>
__global__ void l2l_k(int p, int ls, int le, const int *__restrict__ parent, const int4 *__restrict__ xyz,
                      const T *__restrict__ rtab, T *__restrict__ L)
{
    const int ntri = p * (p + 1) / 2, PP = p * p;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = ls + (int)(gid / ntri);
    const int ci = (int)(gid % ntri);
    if (c >= le) return;
    int k, l;
    tri_inv(ci, k, l);
    const T *R = rtab + (size_t)child_octant(xyz[c]) * PP * 2;
    const T *Lp = L + (size_t)parent[c] * PP;
    T sr = 0, si = 0;
    for (int n = k; n < p; n++) {
        const int d = n - k;
        for (int m = -n; m <= n; m++) {
            const int mu = m - l;
            if (mu > d || mu < -d) continue;
            T lr, li;
            cget(Lp, n, m, lr, li);
            const T rr = R[2 * full(d, mu)], ri = -R[2 * full(d, mu) + 1];
            sr += lr * rr - li * ri;
            si += lr * ri + li * rr;
        }
    }
    const T sc = (T)ldexp(1.0, -(k + 1));
    T *Lc = L + (size_t)c * PP;
    Lc[re_idx(k, l)] += sc * sr;
    if (l) Lc[im_idx(k, l)] += sc * si;
}

// M2M and L2L of the mixed path as dense maps: one warp per cell, lane i
// owns output rows i, i + 32, ... (NR of them); the input expansion is staged
// in shared memory and every lane reads the map column by column (coalesced).
constexpr int MV_WARPS = 8;

// M2M: one block per parent, warp w maps child w; the partial expansions are
// added in child order, so the result does not depend on scheduling
template <int NR>
__global__ void __launch_bounds__(32 * MV_WARPS) m2m_mv_k(int PP, int ls, int le, const int *__restrict__ child,
                                                         const int *__restrict__ nchild, const int4 *__restrict__ xyz,
                                                         const float *__restrict__ mat, float *__restrict__ M)
{
    extern __shared__ float sm_mv[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = ls + blockIdx.x;
    const int nc = nchild[c];
    if (nc == 0) return;  // a leaf keeps its P2M expansion
    float *sx = sm_mv + w * PP;                 // child expansion
    float *part = sm_mv + MV_WARPS * PP;        // [child][PP] partial results
    if (w < nc) {
        const int ch = child[c] + w;
        const float *T = mat + (size_t)child_octant(xyz[ch]) * PP * PP;
        const float *Mc = M + (size_t)ch * PP;
        for (int j = lane; j < PP; j += 32) sx[j] = Mc[j];
        __syncwarp();
        float acc[NR];
#pragma unroll
        for (int r = 0; r < NR; r++) acc[r] = 0.f;
        for (int j = 0; j < PP; j++) {
            const float xj = sx[j];
            const float *col = T + (size_t)j * PP;
#pragma unroll
            for (int r = 0; r < NR; r++) {
                const int i = lane + 32 * r;
                if (i < PP) acc[r] = fmaf(col[i], xj, acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; r++) {
            const int i = lane + 32 * r;
            if (i < PP) part[w * PP + i] = acc[r];
        }
    }
    __syncthreads();
    float *Mp = M + (size_t)c * PP;
    for (int i = threadIdx.x; i < PP; i += 32 * MV_WARPS) {
        float sum = 0.f;
        for (int k = 0; k < nc; k++) sum += part[k * PP + i];
        Mp[i] = sum;
    }
}

// L2L into child c by one warp, sx: PP floats of the warp's shared memory
template <int NR>
__device__ __forceinline__ void l2l_child_warp(int c, int lane, int PP, const int *__restrict__ parent,
                                               const int4 *__restrict__ xyz, const float *__restrict__ mat,
                                               float *__restrict__ L, float *sx)
{
    const float *T = mat + (size_t)child_octant(xyz[c]) * PP * PP;
    const float *Lp = L + (size_t)parent[c] * PP;
    for (int j = lane; j < PP; j += 32) sx[j] = __ldcg(Lp + j);
    __syncwarp();
    float acc[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) acc[r] = 0.f;
    for (int j = 0; j < PP; j++) {
        const float xj = sx[j];
        const float *col = T + (size_t)j * PP;
#pragma unroll
        for (int r = 0; r < NR; r++) {
            const int i = lane + 32 * r;
            if (i < PP) acc[r] = fmaf(col[i], xj, acc[r]);
        }
    }
    float *Lc = L + (size_t)c * PP;
#pragma unroll
    for (int r = 0; r < NR; r++) {
        const int i = lane + 32 * r;
        if (i < PP) Lc[i] = __ldcg(Lc + i) + acc[r];
    }
}

template <int NR>
__global__ void __launch_bounds__(32 * MV_WARPS) l2l_mv_k(int PP, int ls, int le, const int *__restrict__ parent,
                                                         const int4 *__restrict__ xyz, const float *__restrict__ mat,
                                                         float *__restrict__ L)
{
    extern __shared__ float sm_mv[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = ls + blockIdx.x * MV_WARPS + w;
    if (c >= le) return;
    l2l_child_warp<NR>(c, lane, PP, parent, xyz, mat, L, sm_mv + w * PP);
}

// M2M of parent c by one warp, with the arithmetic of m2m_mv_k (each child's
// map in the same order, the children's partial results added in child
// order); sx: PP floats of the warp's shared memory
template <int NR>
__device__ __forceinline__ void m2m_parent_warp(int c, int lane, int PP, const int *__restrict__ child,
                                                const int *__restrict__ nchild, const int4 *__restrict__ xyz,
                                                const float *__restrict__ mat, float *__restrict__ M, float *sx)
{
    const int nc = nchild[c];
    if (nc == 0) return;
    float sum[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) sum[r] = 0.f;
    for (int k = 0; k < nc; k++) {
        const int ch = child[c] + k;
        const float *T = mat + (size_t)child_octant(xyz[ch]) * PP * PP;
        const float *Mc = M + (size_t)ch * PP;
        __syncwarp();
        for (int j = lane; j < PP; j += 32) sx[j] = __ldcg(Mc + j);
        __syncwarp();
        float acc[NR];
#pragma unroll
        for (int r = 0; r < NR; r++) acc[r] = 0.f;
        for (int j = 0; j < PP; j++) {
            const float xj = sx[j];
            const float *col = T + (size_t)j * PP;
#pragma unroll
            for (int r = 0; r < NR; r++) {
                const int i = lane + 32 * r;
                if (i < PP) acc[r] = fmaf(col[i], xj, acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; r++) sum[r] += acc[r];
    }
    float *Mp = M + (size_t)c * PP;
#pragma unroll
    for (int r = 0; r < NR; r++) {
        const int i = lane + 32 * r;
        if (i < PP) Mp[i] = sum[r];
    }
}

static void m2m_mv(int PP, int ls, int le, const int *child, const int *nchild, const int4 *xyz, const float *mat,
                   float *M, cudaStream_t s)
{
    const unsigned g = (unsigned)(le - ls);
    const size_t sm = sizeof(float) * 2 * MV_WARPS * PP;
    switch ((PP + 31) / 32) {
#define FMM_MV_CASE(R) \
    case R: m2m_mv_k<R><<<g, 32 * MV_WARPS, sm, s>>>(PP, ls, le, child, nchild, xyz, mat, M); break;
        FMM_MV_CASE(1) FMM_MV_CASE(2) FMM_MV_CASE(3) FMM_MV_CASE(4) FMM_MV_CASE(5) FMM_MV_CASE(6) FMM_MV_CASE(7)
        FMM_MV_CASE(8) FMM_MV_CASE(9) FMM_MV_CASE(10) FMM_MV_CASE(11) FMM_MV_CASE(12) FMM_MV_CASE(13)
#undef FMM_MV_CASE
    default: throw Error{FMM_EINVAL, "m2m: unsupported p"};
    }
}

static void l2l_mv(int PP, int ls, int le, const int *parent, const int4 *xyz, const float *mat, float *L, cudaStream_t s)
{
    const unsigned g = nblk(le - ls, MV_WARPS);
    const size_t sm = sizeof(float) * MV_WARPS * PP;
    switch ((PP + 31) / 32) {
#define FMM_MV_CASE(R) \
    case R: l2l_mv_k<R><<<g, 32 * MV_WARPS, sm, s>>>(PP, ls, le, parent, xyz, mat, L); break;
        FMM_MV_CASE(1) FMM_MV_CASE(2) FMM_MV_CASE(3) FMM_MV_CASE(4) FMM_MV_CASE(5) FMM_MV_CASE(6) FMM_MV_CASE(7)
        FMM_MV_CASE(8) FMM_MV_CASE(9) FMM_MV_CASE(10) FMM_MV_CASE(11) FMM_MV_CASE(12) FMM_MV_CASE(13)
#undef FMM_MV_CASE
    default: throw Error{FMM_EINVAL, "l2l: unsupported p"};
    }
}

// Column m (orders +m and -m) of I_n^m(u), n = m .. Q-1, written to full
// complex storage sI[2 * (n*n + n +- m)]; computed in FP64 by one thread:
// I_m^m = (2m-1)!! (x + iy)^m / r^(2m+1), then the three-term recurrence in n.
template <class T>
__device__ void irregular_column(int Q, int m, double x, double y, double z, T *sI)
{
    const double r2 = x * x + y * y + z * z, ir2 = 1.0 / r2;
    const double sg = (m & 1) ? -1.0 : 1.0;
    auto put = [&](int n, double cr, double ci) {
        sI[2 * (n * n + n + m)] = (T)cr;
        sI[2 * (n * n + n + m) + 1] = (T)ci;
        if (m) {
            sI[2 * (n * n + n - m)] = (T)(sg * cr);
            sI[2 * (n * n + n - m) + 1] = (T)(-sg * ci);
        }
    };
    double pr = sqrt(ir2), pi = 0.0;  // I_0^0 = 1/r
    for (int k = 1; k <= m; k++) {
        const double f = (double)(2 * k - 1) * ir2;
        const double a = (pr * x - pi * y) * f, b = (pr * y + pi * x) * f;
        pr = a;
        pi = b;
    }
    put(m, pr, pi);
    if (m + 1 >= Q) return;
    const double f1 = (double)(2 * m + 1) * z * ir2;
    double p2r = pr, p2i = pi, p1r = pr * f1, p1i = pi * f1;
    put(m + 1, p1r, p1i);
    for (int n = m + 2; n < Q; n++) {
        const double a = (double)(2 * n - 1) * z, b = (double)((n + m - 1) * (n - m - 1));
        const double cr = (a * p1r - b * p2r) * ir2, ci = (a * p1i - b * p2i) * ir2;
        put(n, cr, ci);
        p2r = p1r;
        p2i = p1i;
        p1r = cr;
        p1i = ci;
    }
}

// ---------------------------------------------------------------------------
// M2L on the CUDA cores, same-level pairs from the octant stencil.
// One block per tile of targets (one level, one octant); the loop runs over
// the stencil vectors v, gathering for each target the source at lattice
// offset v (absent cells contribute nothing).
// ---------------------------------------------------------------------------
constexpr int M2L_CC_T = 128, M2L_CC_ACC = 12, M2L_CC_FLUSH = 16;

template <class T>
struct Acc { using type = double; };

template <class T>
__global__ void __launch_bounds__(M2L_CC_T) m2l_cc_k(int p, const M2LTile *__restrict__ tiles, const int *__restrict__ ntiles,
                                                     const int *__restrict__ tgt, const int4 *__restrict__ xyz,
                                                     const uint64_t *__restrict__ anchor, const LevelDesc *__restrict__ ld,
                                                     const int *__restrict__ map_pool, const int4 *__restrict__ st,
                                                     const int *__restrict__ st_off, const T *__restrict__ M,
                                                     T *__restrict__ L, int tile_max)
{
    if ((int)blockIdx.x >= *ntiles) return;
    const M2LTile td = tiles[blockIdx.x];
    const int PP = p * p, Q = 2 * p - 1, QQ = Q * Q, ntri = p * (p + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sI = reinterpret_cast<T *>(smem_raw);                 // QQ complex
    T *sM = sI + 2 * QQ;                                     // tile_max * PP complex
    int *ssrc = reinterpret_cast<int *>(sM + 2 * (size_t)tile_max * PP);
    int *spos = ssrc + tile_max;                             // 5 per target

    const int l = td.level;
    // per target: lattice position, level and octant (a pooled tile mixes them)
    if ((int)threadIdx.x < td.count) {
        const int4 a = xyz[tgt[td.start + threadIdx.x]];
        const int sh = FMM_MAXLEVEL - a.w;
        int *sp = spos + 5 * threadIdx.x;
        sp[0] = a.x >> sh;
        sp[1] = a.y >> sh;
        sp[2] = a.z >> sh;
        sp[3] = a.w;
        sp[4] = (sp[0] & 1) | ((sp[1] & 1) << 1) | ((sp[2] & 1) << 2);
    }
    const int nout = td.count * ntri;
    using A = typename Acc<T>::type;
    T blk[2 * M2L_CC_ACC];
    A tot[2 * M2L_CC_ACC];
#pragma unroll
    for (int r = 0; r < 2 * M2L_CC_ACC; r++) {
        blk[r] = T(0);
        tot[r] = A(0);
    }
    // the set's entries are sorted by reach: only a prefix can hit a cell
    const int e0 = st_off[td.octant], e1 = e0 + st_off[10 + td.octant * (FMM_MAXLEVEL + 1) + l];
    int since = 0;
    for (int e = e0; e < e1; e++) {
        const int4 v = st[e];
        __syncthreads();
        if ((int)threadIdx.x < td.count) {
            const int *sp = spos + 5 * threadIdx.x;
            ssrc[threadIdx.x] = ((v.w >> (16 + sp[4])) & 1)
                                    ? level_lookup(ld[sp[3]], map_pool, anchor, sp[3], sp[0] + v.x, sp[1] + v.y, sp[2] + v.z)
                                    : -1;
        }
        if ((int)threadIdx.x < Q) irregular_column(Q, (int)threadIdx.x, -(double)v.x, -(double)v.y, -(double)v.z, sI);
        __syncthreads();
        for (int i = threadIdx.x; i < td.count * PP; i += blockDim.x) {
            const int t = i / PP, f = i - t * PP;
            const int src = ssrc[t];
            int j = (int)sqrtf((float)f);
            while (j * j > f) j--;
            while ((j + 1) * (j + 1) <= f) j++;
            const int k = f - j * j - j;
            T re = 0, im = 0;
            if (src >= 0) cget(M + (size_t)src * PP, j, k, re, im);
            sM[2 * ((size_t)t * PP + f)] = re;
            sM[2 * ((size_t)t * PP + f) + 1] = im;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < M2L_CC_ACC; r++) {
            const int o = threadIdx.x + r * M2L_CC_T;
            if (o >= nout) break;
            const int t = o / ntri;
            if (ssrc[t] < 0) continue;
            int n, m;
            tri_inv(o - t * ntri, n, m);
            const T *Mt = sM + 2 * (size_t)t * PP;
            T sr = 0, si = 0;
            for (int j = 0; j < p; j++)
                for (int k = -j; k <= j; k++) {
                    const T mr = Mt[2 * full(j, k)], mi = Mt[2 * full(j, k) + 1];
                    const int fi = full(j + n, k + m);
                    const T ir = sI[2 * fi], ii = sI[2 * fi + 1];
                    sr += mr * ir - mi * ii;
                    si += mr * ii + mi * ir;
                }
            if (n & 1) {
                sr = -sr;
                si = -si;
            }
            blk[2 * r] += sr;
            blk[2 * r + 1] += si;
        }
        if (++since == M2L_CC_FLUSH || e + 1 == e1) {
            since = 0;
#pragma unroll
            for (int r = 0; r < 2 * M2L_CC_ACC; r++) {
                tot[r] += (A)blk[r];
                blk[r] = T(0);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < M2L_CC_ACC; r++) {
        const int o = threadIdx.x + r * M2L_CC_T;
        if (o >= nout) break;
        const int t = o / ntri;
        int n, m;
        tri_inv(o - t * ntri, n, m);
        T *Lc = L + (size_t)tgt[td.start + t] * PP;
        Lc[re_idx(n, m)] += (T)tot[2 * r];
        if (m) Lc[im_idx(n, m)] += (T)tot[2 * r + 1];
    }
}

// ---------------------------------------------------------------------------
// M2L between cells of different levels (explicit list).
//
// With s = max(w_A, w_B) and u = (c_A - c_B) / s, the scaled expansions
// (M~_j = M_j / w_B^j, L~_n = L_n w_A^(n+1)) give
//   L~_n^m += (w_A/s)^(n+1) (-1)^n sum_{j,k} (w_B/s)^j M~_j^k I_{j+n}^{k+m}(u).
// Both ratios are powers of two no larger than 1 and |u| stays above the
// acceptance distance, so nothing overflows in FP32 whatever the level gap
// (terms of a cell many levels smaller than its partner underflow to zero,
// their true size).  One block of four warps per target cell; warp w takes
// the cell's pairs w, w + 4, ...: lanes 0..Q-1 build one column m of I(u)
// each, the warp gathers the source's M~, then lane o owns outputs o and
// o + 32 of the triangle.  The four warp sums are added in warp order.
// ---------------------------------------------------------------------------
constexpr int M2LX_W = 4;

// Column m of I_n^m(u), n = m .. Q-1, computed in C and written as T to
// complex storage whose entry (n, m) sits at row(n) + m (full storage: row(n)
// = n^2 + n): I_m^m = (2m-1)!! (x + iy)^m / r^(2m+1), then the three-term
// recurrence in n; orders -m from I_n^-m = (-1)^m conj(I_n^m).
struct FullRows {
    __device__ int operator()(int n) const { return n * n + n; }
};

template <class C, class T, class Row = FullRows>
__device__ void irregular_col(int Q, int m, C x, C y, C z, T *sI, Row row = Row())
{
    const C r2 = x * x + y * y + z * z, ir2 = C(1) / r2;
    const C sg = (m & 1) ? C(-1) : C(1);
    auto put = [&](int n, C cr, C ci) {
        const int e = row(n);
        sI[2 * (e + m)] = (T)cr;
        sI[2 * (e + m) + 1] = (T)ci;
        if (m) {
            sI[2 * (e - m)] = (T)(sg * cr);
            sI[2 * (e - m) + 1] = (T)(-sg * ci);
        }
    };
    C pr = sqrt(ir2), pi = C(0);
    for (int k = 1; k <= m; k++) {
        const C f = C(2 * k - 1) * ir2;
        const C a = (pr * x - pi * y) * f, b = (pr * y + pi * x) * f;
        pr = a;
        pi = b;
    }
    put(m, pr, pi);
    if (m + 1 >= Q) return;
    const C f1 = C(2 * m + 1) * z * ir2;
    C p2r = pr, p2i = pi, p1r = pr * f1, p1i = pi * f1;
    put(m + 1, p1r, p1i);
    for (int n = m + 2; n < Q; n++) {
        const C a = C(2 * n - 1) * z, b = C((n + m - 1) * (n - m - 1));
        const C cr = (a * p1r - b * p2r) * ir2, ci = (a * p1i - b * p2i) * ir2;
        put(n, cr, ci);
        p2r = p1r;
        p2i = p1i;
        p1r = cr;
        p1i = ci;
    }
}

template <class T>
__global__ void __launch_bounds__(32 * M2LX_W) m2lx_k(int p, int nc, const int *__restrict__ ptr,
                                                      const int *__restrict__ src, const int4 *__restrict__ xyz,
                                                      const T *__restrict__ M, T *__restrict__ L)
{
    const int c = blockIdx.x;
    if (c >= nc) return;
    const int k0 = ptr[c], k1 = ptr[c + 1];
    if (k0 == k1) return;
    const int PP = p * p, Q = 2 * p - 1, ntri = p * (p + 1) / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // per warp: its running sums (2 ntri FP64), I(u) (Q*Q complex), M~ (PP complex)
    double *sA = reinterpret_cast<double *>(smem_raw) + (size_t)warp * 2 * ntri;
    T *sI = reinterpret_cast<T *>(smem_raw + sizeof(double) * M2LX_W * 2 * ntri) + (size_t)warp * 2 * (Q * Q + PP);
    T *sM = sI + 2 * Q * Q;
    for (int o = lane; o < 2 * ntri; o += 32) sA[o] = 0.0;
    const int4 a = xyz[c];
    const long long WA = 1LL << (FMM_MAXLEVEL - a.w);
    for (int k = k0 + warp; k < k1; k += M2LX_W) {
        const int B = src[k];
        const int4 b = xyz[B];
        const long long WB = 1LL << (FMM_MAXLEVEL - b.w);
        const int dl = a.w - b.w;  // > 0: the target is the smaller cell
        // u = (c_A - c_B) / max(w_A, w_B) from half-grid units; exact in FP64
        const double sc = 1.0 / (double)(2 * (WA > WB ? WA : WB));
        const double ux = (double)(2LL * (a.x - b.x) + (WA - WB)) * sc;
        const double uy = (double)(2LL * (a.y - b.y) + (WA - WB)) * sc;
        const double uz = (double)(2LL * (a.z - b.z) + (WA - WB)) * sc;
        __syncwarp();
        for (int m = lane; m < Q; m += 32) irregular_col<T, T>(Q, m, (T)ux, (T)uy, (T)uz, sI);
        for (int i = lane; i < PP; i += 32) {
            int j = (int)sqrtf((float)i);
            while (j * j > i) j--;
            while ((j + 1) * (j + 1) <= i) j++;
            const int kk = i - j * j - j;
            T re, im;
            cget(M + (size_t)B * PP, j, kk, re, im);
            const T f = dl < 0 ? (T)ldexp(1.0, dl * j) : T(1);  // (w_B / s)^j
            sM[2 * i] = re * f;
            sM[2 * i + 1] = im * f;
        }
        __syncwarp();
        for (int o = lane; o < ntri; o += 32) {
            int n, m;
            tri_inv(o, n, m);
            T sr = 0, si = 0;
            for (int j = 0; j < p; j++)
                for (int kk = -j; kk <= j; kk++) {
                    const T mr = sM[2 * full(j, kk)], mi = sM[2 * full(j, kk) + 1];
                    const int fi = full(j + n, kk + m);
                    const T ir = sI[2 * fi], ii = sI[2 * fi + 1];
                    sr += mr * ir - mi * ii;
                    si += mr * ii + mi * ir;
                }
            double f = dl > 0 ? ldexp(1.0, -dl * (n + 1)) : 1.0;  // (w_A / s)^(n+1)
            if (n & 1) f = -f;
            sA[2 * o] += f * (double)sr;
            sA[2 * o + 1] += f * (double)si;
        }
    }
    __syncthreads();
    if (warp) return;
    const double *sA0 = reinterpret_cast<const double *>(smem_raw);
    T *Lc = L + (size_t)c * PP;
    for (int o = lane; o < ntri; o += 32) {
        int n, m;
        tri_inv(o, n, m);
        double sr = 0, si = 0;
        for (int w = 0; w < M2LX_W; w++) {
            sr += sA0[(size_t)w * 2 * ntri + 2 * o];
            si += sA0[(size_t)w * 2 * ntri + 2 * o + 1];
        }
        Lc[re_idx(n, m)] += (T)sr;
        if (m) Lc[im_idx(n, m)] += (T)si;
    }
}

// FP32 form of the same for p = 2 .. 10, p fixed at compile time. Eight warps
// per target cell, each half-warp on its own pair: the cell's pair q goes to
// half-warp q % 16. Lane u of a half-warp owns a run of R consecutive orders
// m0 .. m0+R-1 of one degree n (M2lxLayout<P>), so each entry of I(u) it loads
// serves up to R outputs and each row of M~ it loads (16-byte broadcast loads)
// serves R; the rows of I(u) are placed so that the 16 lanes' loads of one
// step fall in 16 different bank pairs (m2lx_layout.py gives the argument).
// A warp loads the source ids and cells of 32 of its pairs at once (lane i:
// pair i), prefetches each half's next M~ while the current pair is computed,
// and keeps running sums as FP32 (hi, lo) pairs; the 16 partial sums are added
// in half-warp order.
constexpr int M2LX_FW = 8;

__device__ __forceinline__ void m2lx_two_sum(float &hi, float &lo, float b)
{
    const float s = hi + b;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}

// entry of I_l^0 in a half-warp's table: row l starts where row l-1 ends,
// moved up to the first entry with rowptr(l) = C l (mod 16)
template <int P>
__host__ __device__ constexpr int m2lx_rowptr(int l)
{
    int nxt = 0, b = 0;
    for (int i = 0; i <= l; i++) {
        b = nxt;
        while ((((b + i - M2lxLayout<P>::C * i) % 16) + 16) % 16 != 0) b++;
        nxt = b + 2 * i + 1;
    }
    return b + l;
}

// entries of one half-warp's I table (the last row, the R-1 entries a run
// reads past its end), rounded up to even so that M~ starts 16-byte aligned
template <int P>
__host__ __device__ constexpr int m2lx_isize()
{
    constexpr int Q = 2 * P - 1;
    return (m2lx_rowptr<P>(Q - 1) + Q + M2lxLayout<P>::R - 1 + 1) & ~1;
}

template <int P>
constexpr size_t m2lx_f_smem()
{
    // per half-warp: I table, then M~ rows j at j(j+1) (2j+1 entries and one
    // spare, so each row is whole 16-byte pairs); the partial sums; the row table
    return sizeof(float2) * 2 * M2LX_FW * (size_t)(m2lx_isize<P>() + P * (P + 1)) +
           sizeof(double) * 2 * M2LX_FW * (size_t)(P * (P + 1)) + sizeof(int) * 2 * P;
}

struct TableRows {
    const int *rp;
    __device__ int operator()(int n) const { return rp[n]; }
};

// different-level M2L into target cell c by one CTA of 32 M2LX_FW threads
template <int P>
__device__ __forceinline__ void m2lx_f_cell(int c, const int *__restrict__ ptr, const int *__restrict__ src,
                                            const int4 *__restrict__ xyz, const float *__restrict__ M,
                                            float *__restrict__ L, unsigned char *smem_raw)
{
    using Lay = M2lxLayout<P>;
    constexpr int PP = P * P, Q = 2 * P - 1, NT = P * (P + 1) / 2, NM = (PP + 15) / 16, R = Lay::R;
    constexpr int NH = 2 * M2LX_FW;  // half-warps
    constexpr int IS = m2lx_isize<P>(), HS = IS + P * (P + 1);
    const int k0 = ptr[c], npair = ptr[c + 1] - k0;
    if (npair == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const int hw = 2 * warp + half;
    float2 *sI = reinterpret_cast<float2 *>(smem_raw) + (size_t)hw * HS;
    float2 *sM = sI + IS;
    double *red = reinterpret_cast<double *>(reinterpret_cast<float2 *>(smem_raw) + (size_t)NH * HS);
    int *rp = reinterpret_cast<int *>(red + (size_t)NH * 2 * NT);
    if ((int)threadIdx.x < Q) rp[threadIdx.x] = m2lx_rowptr<P>((int)threadIdx.x);
    __syncthreads();
    const int4 a = xyz[c];
    // this lane's entries of M~ in full complex storage: i = hl + 16 r = j^2 + j + k,
    // staged at j(j+1) + j + k = i + j
    int mre[NM], mim[NM], mj[NM];
    float msr[NM], msi[NM];
#pragma unroll
    for (int r = 0; r < NM; r++) {
        const int i = hl + 16 * r;
        int j = 0;
        while ((j + 1) * (j + 1) <= i) j++;
        const int k = i - j * j - j, ak = k < 0 ? -k : k;
        mj[r] = j;
        mre[r] = i < PP ? j * j + (ak ? 2 * ak - 1 : 0) : 0;
        mim[r] = i < PP && ak ? j * j + 2 * ak : -1;
        // X_j^-k = (-1)^k conj(X_j^k)
        const float sg = (k < 0 && (ak & 1)) ? -1.f : 1.f;
        msr[r] = sg;
        msi[r] = k < 0 ? -sg : sg;
    }
    // this lane's run of outputs: degree rn, orders rm0 .. rm0 + rlen - 1
    const int rn = (int)((Lay::N >> (4 * hl)) & 15ull), rm0 = (int)((Lay::M0 >> (4 * hl)) & 15ull),
              rlen = (int)((Lay::LEN >> (4 * hl)) & 15ull);
    // step t of row j reads I entry ib[j] + t
    int ib[P];
#pragma unroll
    for (int j = 0; j < P; j++) ib[j] = rlen ? rp[j + rn] + rm0 - j : 0;
    float ahr[R], alr[R], ahi[R], ali[R];
#pragma unroll
    for (int i = 0; i < R; i++) ahr[i] = alr[i] = ahi[i] = ali[i] = 0.f;

    // step t of this warp: half h takes pair q = NH t + 2 warp + h
    const int nstep = npair > 2 * warp ? (npair - 2 * warp + NH - 1) / NH : 0;
    float pre[NM], pim[NM];
    auto fetch = [&](int B) {
#pragma unroll
        for (int r = 0; r < NM; r++) {
            pre[r] = hl + 16 * r < PP ? M[(size_t)B * PP + mre[r]] : 0.f;
            pim[r] = hl + 16 * r < PP && mim[r] >= 0 ? M[(size_t)B * PP + mim[r]] : 0.f;
        }
    };
    for (int t0 = 0; t0 < nstep; t0 += 16) {
        const int nb = min(16, nstep - t0);
        int Bl = 0;
        int4 bl = make_int4(0, 0, 0, 0);
        {
            const int q = NH * (t0 + (lane >> 1)) + 2 * warp + (lane & 1);
            if ((lane >> 1) < nb && q < npair) {
                Bl = src[k0 + q];
                bl = xyz[Bl];
            }
        }
        {
            const int B0 = __shfl_sync(0xffffffffu, Bl, half);
            if (NH * t0 + 2 * warp + half < npair) fetch(B0);
        }
        for (int t = 0; t < nb; t++) {
            const int li = 2 * t + half;  // lane holding this half's pair
            const bool valid = NH * (t0 + t) + 2 * warp + half < npair;
            const int bw = __shfl_sync(0xffffffffu, bl.w, li);
            const int bx = __shfl_sync(0xffffffffu, bl.x, li), by = __shfl_sync(0xffffffffu, bl.y, li),
                      bz = __shfl_sync(0xffffffffu, bl.z, li);
            const int Bn = __shfl_sync(0xffffffffu, Bl, min(li + 2, 31));
            const int dl = a.w - bw;  // > 0: the target is the smaller cell
            const int lmin = a.w < bw ? a.w : bw;
            const long long WA = 1LL << (FMM_MAXLEVEL - a.w), WB = 1LL << (FMM_MAXLEVEL - bw);
            // u = (c_A - c_B) / max(w_A, w_B): integers below 2^24 times a power of two, exact in FP32
            const float sc = ldexpf(1.f, -(FMM_MAXLEVEL + 1 - lmin));
            const float ux = (float)(2LL * (a.x - bx) + (WA - WB)) * sc;
            const float uy = (float)(2LL * (a.y - by) + (WA - WB)) * sc;
            const float uz = (float)(2LL * (a.z - bz) + (WA - WB)) * sc;
            __syncwarp();
            if (valid) {
                for (int m = hl; m < Q; m += 16)
                    irregular_col<float, float>(Q, m, ux, uy, uz, reinterpret_cast<float *>(sI), TableRows{rp});
#pragma unroll
                for (int r = 0; r < NM; r++)
                    if (hl + 16 * r < PP) {
                        const float f = dl < 0 ? ldexpf(1.f, dl * mj[r]) : 1.f;  // (w_B / s)^j
                        sM[hl + 16 * r + mj[r]] = make_float2(pre[r] * msr[r] * f, pim[r] * msi[r] * f);
                    }
            }
            if (t + 1 < nb && NH * (t0 + t + 1) + 2 * warp + half < npair) fetch(Bn);
            __syncwarp();
            if (!valid || rlen == 0) continue;
            // four partial sums per output (the four real products) keep the
            // FMA chains independent
            float a0[R], a1[R], a2[R], a3[R];
#pragma unroll
            for (int i = 0; i < R; i++) a0[i] = a1[i] = a2[i] = a3[i] = 0.f;
#pragma unroll
            for (int j = 0; j < P; j++) {
                float2 mv[2 * P];
                const float4 *Mj = reinterpret_cast<const float4 *>(sM + j * (j + 1));
#pragma unroll
                for (int s2 = 0; s2 <= j; s2++) {
                    const float4 v = Mj[s2];
                    mv[2 * s2] = make_float2(v.x, v.y);
                    mv[2 * s2 + 1] = make_float2(v.z, v.w);
                }
                const float2 *Ij = sI + ib[j];
#pragma unroll
                for (int e = 0; e < 2 * j + R; e++) {
                    const float2 iv = Ij[e];
#pragma unroll
                    for (int i = 0; i < R; i++) {
                        const int k = e - i - j;  // output m = rm0 + i takes I_{j+n}^{m+k} M_j^k
                        if (k >= -j && k <= j) {
                            const float2 mk = mv[k + j];
                            a0[i] = fmaf(mk.x, iv.x, a0[i]);
                            a1[i] = fmaf(mk.y, iv.y, a1[i]);
                            a2[i] = fmaf(mk.x, iv.y, a2[i]);
                            a3[i] = fmaf(mk.y, iv.x, a3[i]);
                        }
                    }
                }
            }
            float f = dl > 0 ? ldexpf(1.f, -dl * (rn + 1)) : 1.f;  // (w_A / s)^(n+1)
            if (rn & 1) f = -f;
#pragma unroll
            for (int i = 0; i < R; i++) {
                m2lx_two_sum(ahr[i], alr[i], f * (a0[i] - a1[i]));
                m2lx_two_sum(ahi[i], ali[i], f * (a2[i] + a3[i]));
            }
        }
    }
    const int o0 = rn * (rn + 1) / 2 + rm0;
#pragma unroll
    for (int i = 0; i < R; i++)
        if (i < rlen) {
            red[(size_t)hw * 2 * NT + 2 * (o0 + i)] = (double)ahr[i] + (double)alr[i];
            red[(size_t)hw * 2 * NT + 2 * (o0 + i) + 1] = (double)ahi[i] + (double)ali[i];
        }
    __syncthreads();
    if (warp) return;
    float *Lc = L + (size_t)c * PP;
    for (int o = lane; o < NT; o += 32) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= o) n++;
        const int m = o - n * (n + 1) / 2;
        double sr = 0, si = 0;
        for (int w = 0; w < NH; w++) {  // every half-warp wrote all its outputs (zero without pairs)
            sr += red[(size_t)w * 2 * NT + 2 * o];
            si += red[(size_t)w * 2 * NT + 2 * o + 1];
        }
        Lc[re_idx(n, m)] += (float)sr;
        if (m) Lc[im_idx(n, m)] += (float)si;
    }
}

template <int P>
__global__ void __launch_bounds__(32 * M2LX_FW, 2) m2lx_f_k(int nc, const int *__restrict__ ptr,
                                                            const int *__restrict__ src, const int4 *__restrict__ xyz,
                                                            const float *__restrict__ M, float *__restrict__ L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if ((int)blockIdx.x >= nc) return;
    m2lx_f_cell<P>((int)blockIdx.x, ptr, src, xyz, M, L, smem_raw);
}

template <int P>
static void m2lx_f_run(int nc, const int *ptr, const int *src, const int4 *xyz, const float *M, float *L, cudaStream_t s)
{
    constexpr size_t smem = m2lx_f_smem<P>();
    ensure_smem((const void *)m2lx_f_k<P>, smem);
    m2lx_f_k<P><<<nc, 32 * M2LX_FW, smem, s>>>(nc, ptr, src, xyz, M, L);
}

static bool m2lx_f_launch(int p, int nc, const int *ptr, const int *src, const int4 *xyz, const float *M, float *L,
                          cudaStream_t s)
{
    switch (p) {
#define FMM_M2LX_CASE(PV) \
    case PV: m2lx_f_run<PV>(nc, ptr, src, xyz, M, L, s); return true;
        FMM_M2LX_CASE(2) FMM_M2LX_CASE(3) FMM_M2LX_CASE(4) FMM_M2LX_CASE(5) FMM_M2LX_CASE(6)
        FMM_M2LX_CASE(7) FMM_M2LX_CASE(8) FMM_M2LX_CASE(9) FMM_M2LX_CASE(10)
#undef FMM_M2LX_CASE
    default: return false;
    }
}

// ---------------------------------------------------------------------------
// L2P: one block per leaf; phi and grad of the far field into far[] (sorted)
// ---------------------------------------------------------------------------
template <class T, class P4>
__global__ void __launch_bounds__(64) l2p_k(int p, const int *__restrict__ leaves, const int *__restrict__ begin,
                                            const int *__restrict__ end, const int4 *__restrict__ xyz,
                                            const Box *__restrict__ box, const P4 *__restrict__ xs,
                                            const T *__restrict__ L, double4_32a *__restrict__ far)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sL = reinterpret_cast<T *>(smem_raw);
    const int PP = p * p;
    const int c = leaves[blockIdx.x];
    for (int i = threadIdx.x; i < PP; i += blockDim.x) sL[i] = L[(size_t)c * PP + i];
    __syncthreads();
    double cen[3], w;
    cell_geom(box, xyz[c], cen, w);
    const double iw = 1.0 / w;
    for (int j = begin[c] + threadIdx.x; j < end[c]; j += blockDim.x) {
        const double4_32a pt = rel_pt(xs, j, cen);
        const T x = (T)(pt.x * iw), y = (T)(pt.y * iw), z = (T)(pt.z * iw);
        const T r2 = x * x + y * y + z * z;
        T F = 0, Fz = 0, Gr = 0, Gi = 0;
        T mre = 1, mim = 0;
        for (int m = 0; m < p; m++) {
            if (m > 0) {
                const T f = T(1) / T(2 * m);
                const T a = (mre * x - mim * y) * f, b = (mre * y + mim * x) * f;
                mre = a;
                mim = b;
            }
            const T wm = m ? T(2) : T(1);
            T p2re = 0, p2im = 0, p1re = 0, p1im = 0;
            for (int n = m; n < p; n++) {
                T rre, rim;
                if (n == m) {
                    rre = mre;
                    rim = mim;
                } else if (n == m + 1) {
                    rre = z * mre;
                    rim = z * mim;
                } else {
                    const T a = T(2 * n - 1), b = T(1) / T((n + m) * (n - m));
                    rre = (a * z * p1re - r2 * p2re) * b;
                    rim = (a * z * p1im - r2 * p2im) * b;
                }
                p2re = p1re; p2im = p1im; p1re = rre; p1im = rim;
                // phi: Re(L_n^m conj(R_n^m)), doubled for m > 0
                const T lr = sL[re_idx(n, m)], li = m ? sL[im_idx(n, m)] : T(0);
                F += wm * (lr * rre + li * rim);
                if (n + 1 < p) {
                    // d/dz: Re(L_{n+1}^m conj(R_n^m)), doubled for m > 0
                    const T zr = sL[re_idx(n + 1, m)], zi = m ? sL[im_idx(n + 1, m)] : T(0);
                    Fz += wm * (zr * rre + zi * rim);
                    // G = (d_x - i d_y) phi: -L_{n+1}^{m-1} conj(R) ...
                    T ar, ai;
                    if (m == 0) {
                        ar = -sL[re_idx(n + 1, 1)];
                        ai = sL[im_idx(n + 1, 1)];
                    } else {
                        ar = sL[re_idx(n + 1, m - 1)];
                        ai = (m - 1) ? sL[im_idx(n + 1, m - 1)] : T(0);
                    }
                    Gr -= ar * rre + ai * rim;
                    Gi -= ai * rre - ar * rim;
                    // ... + conj(L_{n+1}^{m+1} conj(R)) for m >= 1
                    if (m >= 1) {
                        const T br = sL[re_idx(n + 1, m + 1)], bi = sL[im_idx(n + 1, m + 1)];
                        Gr += br * rre + bi * rim;
                        Gi -= bi * rre - br * rim;
                    }
                }
            }
        }
        const double iw2 = iw * iw;
        far[j] = make_double4_32a((double)F * iw, (double)Gr * iw2, -(double)Gi * iw2, (double)Fz * iw2);
    }
}

// geometric centre and inverse width of every cell (cell_geom), once per evaluation
__global__ void cgeo_k(int nc, const int4 *__restrict__ xyz, const Box *__restrict__ box, double4_32a *__restrict__ g)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double cen[3], w;
    cell_geom(box, xyz[c], cen, w);
    g[c] = make_double4_32a(cen[0], cen[1], cen[2], 1.0 / w);
}

// L2P with the order fixed at compile time: one thread per sorted particle,
// the local expansion of its leaf read through the L1 cache (the particles of
// a leaf are consecutive, so a warp reads one or two expansions). The same
// sums as l2p_k: phi = Re sum L_n^m conj(R_n^m), d/dz from L_{n+1}^m and
// (d_x - i d_y) from L_{n+1}^{m-1} and L_{n+1}^{m+1} (Sec. 2.1, L2P).
// L2P of sorted particle j (its leaf c). COHERENT: the local expansion may
// have been written in the same launch by another SM, so it is read through
// L2 (ld.cg) rather than the non-coherent read-only path.
template <int P, class P4, bool COHERENT = false>
__device__ __forceinline__ void l2p_particle(int64_t j, int c, const double4_32a *__restrict__ cgeo,
                                             const P4 *__restrict__ xs, const float *__restrict__ L,
                                             double4_32a *__restrict__ far)
{
    const double4_32a g = cgeo[c];
    const double cen[3] = {g.x, g.y, g.z};
    const double iw = g.w;
    const double4_32a pt = rel_pt(xs, (int)j, cen);
    const float x = (float)(pt.x * iw), y = (float)(pt.y * iw), z = (float)(pt.z * iw);
    const float r2 = x * x + y * y + z * z;
    const float *Lc = L + (size_t)c * (P * P);
    auto ld = [&](int k) { return COHERENT ? __ldcg(Lc + k) : __ldg(Lc + k); };
    float F = 0.f, Fz = 0.f, Gr = 0.f, Gi = 0.f;
    float mre = 1.f, mim = 0.f;
#pragma unroll
    for (int m = 0; m < P; m++) {
        if (m > 0) {
            const float f = 1.f / (float)(2 * m);
            const float a = (mre * x - mim * y) * f, b = (mre * y + mim * x) * f;
            mre = a;
            mim = b;
        }
        const float wm = m ? 2.f : 1.f;
        float p2re = 0.f, p2im = 0.f, p1re = 0.f, p1im = 0.f;
#pragma unroll
        for (int nn = m; nn < P; nn++) {
            float rre, rim;
            if (nn == m) {
                rre = mre;
                rim = mim;
            } else if (nn == m + 1) {
                rre = z * mre;
                rim = z * mim;
            } else {
                const float a = (float)(2 * nn - 1), b = 1.f / (float)((nn + m) * (nn - m));
                rre = (a * z * p1re - r2 * p2re) * b;
                rim = (a * z * p1im - r2 * p2im) * b;
            }
            p2re = p1re; p2im = p1im; p1re = rre; p1im = rim;
            const float lr = ld(re_idx(nn, m)), li = m ? ld(im_idx(nn, m)) : 0.f;
            F += wm * (lr * rre + li * rim);
            if (nn + 1 < P) {
                const float zr = ld(re_idx(nn + 1, m)), zi = m ? ld(im_idx(nn + 1, m)) : 0.f;
                Fz += wm * (zr * rre + zi * rim);
                float ar, ai;
                if (m == 0) {
                    ar = -ld(re_idx(nn + 1, 1));
                    ai = ld(im_idx(nn + 1, 1));
                } else {
                    ar = ld(re_idx(nn + 1, m - 1));
                    ai = (m - 1) ? ld(im_idx(nn + 1, m - 1)) : 0.f;
                }
                Gr -= ar * rre + ai * rim;
                Gi -= ai * rre - ar * rim;
                if (m >= 1) {
                    const float br = ld(re_idx(nn + 1, m + 1)), bi = ld(im_idx(nn + 1, m + 1));
                    Gr += br * rre + bi * rim;
                    Gi -= bi * rre - br * rim;
                }
            }
        }
    }
    const double iw2 = iw * iw;
    far[j] = make_double4_32a((double)F * iw, (double)Gr * iw2, -(double)Gi * iw2, (double)Fz * iw2);
}

template <int P, class P4>
__global__ void __launch_bounds__(256) l2p_flat_k(int64_t n, const int *__restrict__ pcell,
                                                  const double4_32a *__restrict__ cgeo, const P4 *__restrict__ xs,
                                                  const float *__restrict__ L, double4_32a *__restrict__ far)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    l2p_particle<P, P4>(j, pcell[j], cgeo, xs, L, far);
}

template <class P4>
static bool l2p_flat_launch(int p, int64_t n, const int *pcell, const double4_32a *cgeo, const P4 *xs, const float *L,
                            double4_32a *far, cudaStream_t s)
{
    const unsigned g = nblk(n, 256);
    switch (p) {
#define FMM_L2P_CASE(PV) \
    case PV: l2p_flat_k<PV, P4><<<g, 256, 0, s>>>(n, pcell, cgeo, xs, L, far); return true;
        FMM_L2P_CASE(2) FMM_L2P_CASE(3) FMM_L2P_CASE(4) FMM_L2P_CASE(5) FMM_L2P_CASE(6)
        FMM_L2P_CASE(7) FMM_L2P_CASE(8) FMM_L2P_CASE(9) FMM_L2P_CASE(10)
#undef FMM_L2P_CASE
    default: return false;
    }
}

// ---------------------------------------------------------------------------
// host: tables and orchestration
// ---------------------------------------------------------------------------
static int floordiv2(int a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }

int m2l_tile_size(fmm_ctx *h)
{
    if (h->precision == FMM_MIXED && h->engine_used == FMM_M2L_TENSOR) return 128;
    if (h->engine_used == FMM_M2L_ROTATION) return rotation_tile_rows(h);
    const int ntri = h->p * (h->p + 1) / 2;
    int t = std::min(32, (M2L_CC_T * M2L_CC_ACC) / ntri);
    return std::max(t, 1);
}

// Same-level M2L stencils (Sec. 2.1 near/far split under the theta MAC): for
// a target in octant o of its parent, the lattice offsets v with
// 3 < fl(theta^2 |v|^2) (the MAC accepts the pair) whose parent offset
// u = floor((o + v) / 2) has 3 >= fl(theta^2 |u|^2) (the parents were
// rejected). Offsets are bounded by the largest coordinate difference of two
// existing cells of one level, so a tiny theta stays small on shallow trees
// and on deep chains of a few cells alike. Rebuilt only when the bound grows.
static int stencil_reach(const std::array<int, 4> &v)
{
    return std::max(std::abs(v[0]), std::max(std::abs(v[1]), std::abs(v[2])));
}

void stencil_update(fmm_ctx *h)
{
    const double c = h->cmac;
    const int Rfull = 2 * (int)std::ceil(std::sqrt(3.0 / c)) + 3;
    const int R = std::min(Rfull, h->lattice_extent);
    if (R <= h->st_R && h->st_dev.p) return;
    std::map<std::tuple<int, int, int>, int> vid;
    int nv = 0;
    h->st_off.assign(10, 0);
    h->st_host.clear();
    for (int o = 0; o < 8; o++) {
        const int ox = o & 1, oy = (o >> 1) & 1, oz = (o >> 2) & 1;
        for (int vx = -R; vx <= R; vx++)
            for (int vy = -R; vy <= R; vy++)
                for (int vz = -R; vz <= R; vz++) {
                    const double d2 = (double)vx * vx + (double)vy * vy + (double)vz * vz;
                    if (!(3.0 < c * d2)) continue;
                    const int ux = floordiv2(ox + vx), uy = floordiv2(oy + vy), uz = floordiv2(oz + vz);
                    const double u2 = (double)ux * ux + (double)uy * uy + (double)uz * uz;
                    if (3.0 < c * u2) continue;
                    auto key = std::make_tuple(vx, vy, vz);
                    auto it = vid.find(key);
                    int id = it == vid.end() ? (vid[key] = nv++) : it->second;
                    h->st_host.insert(h->st_host.end(), {vx, vy, vz, id});
                }
        h->st_off[o + 1] = (int)(h->st_host.size() / 4);
        // shortest offsets first (stable; the vector ids keep their numbering):
        // a level whose cells span at most E lattice steps reaches only the
        // entries with max(|vx|, |vy|, |vz|) <= E, a prefix of the octant
        std::vector<std::array<int, 4>> eo((size_t)(h->st_off[o + 1] - h->st_off[o]));
        for (size_t i = 0; i < eo.size(); i++)
            for (int k = 0; k < 4; k++) eo[i][k] = h->st_host[4 * ((size_t)h->st_off[o] + i) + k];
        std::stable_sort(eo.begin(), eo.end(), [](const std::array<int, 4> &a, const std::array<int, 4> &b) {
            return stencil_reach(a) < stencil_reach(b);
        });
        for (size_t i = 0; i < eo.size(); i++)
            for (int k = 0; k < 4; k++) h->st_host[4 * ((size_t)h->st_off[o] + i) + k] = eo[i][k];
    }
    if (nv > 0xffff) throw Error{FMM_EINVAL, "M2L stencil: more than 65535 distinct vectors"};
    h->nV = nv;
    // the union of the 8 stencils (each vector once, shortest first) for
    // tiles that pool cells of every octant; bits 16 + o of the fourth int
    // say whether octant o's stencil holds the vector (all 8 bits for the
    // entries of the per-octant lists)
    const int ne8 = h->st_off[8];
    std::vector<std::array<int, 4>> un((size_t)nv);
    for (int e = 0; e < ne8; e++) {
        int *v = &h->st_host[4 * (size_t)e];
        const int o = (int)(std::upper_bound(h->st_off.begin(), h->st_off.begin() + 9, e) - h->st_off.begin()) - 1;
        std::array<int, 4> &u = un[(size_t)v[3]];
        if (!(u[3] >> 16)) u = {v[0], v[1], v[2], v[3]};
        u[3] |= 1 << (16 + o);
        v[3] |= 0xff << 16;
    }
    std::stable_sort(un.begin(), un.end(), [](const std::array<int, 4> &a, const std::array<int, 4> &b) {
        return stencil_reach(a) < stencil_reach(b);
    });
    for (const auto &u : un) h->st_host.insert(h->st_host.end(), {u[0], u[1], u[2], u[3]});
    h->st_off[9] = (int)(h->st_host.size() / 4);
    const int ne = h->st_off[9];
    std::vector<int> buf(4 * (size_t)ne + 10 + 9 * (FMM_MAXLEVEL + 1));
    std::copy(h->st_host.begin(), h->st_host.end(), buf.begin());
    for (int o = 0; o < 10; o++) buf[4 * (size_t)ne + o] = h->st_off[o];
    for (int o = 0; o < 9; o++)
        for (int l = 0; l <= FMM_MAXLEVEL; l++)
            buf[4 * (size_t)ne + 10 + o * (FMM_MAXLEVEL + 1) + l] = h->st_off[o + 1] - h->st_off[o];
    h->st_dev.ensure(sizeof(int) * buf.size());
    FMM_CUDA_TRY(cudaMemcpy(h->st_dev.p, buf.data(), sizeof(int) * buf.size(), cudaMemcpyHostToDevice));
    h->st_R = R;
    // P2P sources of a leaf in a uniform tree: the offsets the MAC rejects
    int near = 0;
    for (int vx = -R; vx <= R; vx++)
        for (int vy = -R; vy <= R; vy++)
            for (int vz = -R; vz <= R; vz++)
                if (!(3.0 < c * ((double)vx * vx + (double)vy * vy + (double)vz * vz))) near++;
    h->p2p_cap_hint = near;
}

void stencil_levels(fmm_ctx *h, cudaStream_t s)
{
    const int ne = h->st_off[9];
    std::vector<int> cnt(9 * (FMM_MAXLEVEL + 1));
    int ecum = -1;
    for (int l = 0; l <= FMM_MAXLEVEL; l++) {
        // no extent known: every entry; an empty level (-1): none
        const int E = l < (int)h->lvl_ext.size() ? h->lvl_ext[l] : INT_MAX;
        ecum = std::max(ecum, E);  // pooled tiles hold cells of this level and above it
        for (int o = 0; o < 9; o++) {
            const int Eo = o < 8 ? E : ecum;
            int e = h->st_off[o];
            while (e < h->st_off[o + 1]) {
                const int *v = &h->st_host[4 * (size_t)e];
                if (std::max(std::abs(v[0]), std::max(std::abs(v[1]), std::abs(v[2]))) > Eo) break;
                e++;
            }
            cnt[o * (FMM_MAXLEVEL + 1) + l] = e - h->st_off[o];
        }
    }
    int *dst = const_cast<int *>(stencil_offsets(h)) + 10;
    FMM_CUDA_TRY(cudaMemcpyAsync(dst, cnt.data(), sizeof(int) * cnt.size(), cudaMemcpyHostToDevice, s));
}

const int *stencil_offsets(fmm_ctx *h)
{
    return reinterpret_cast<const int *>(h->st_dev.as<char>() + sizeof(int4) * h->st_off[9]);
}

// R_n^m(t_o) for the 8 child offsets t_o = (c_child - c_parent) / w_parent
// = (+-1/4, +-1/4, +-1/4), full complex storage, FP64 and FP32 copies.
void operators_init(fmm_ctx *h)
{
    const int p = h->p, PP = p * p;
    std::vector<double> tre(p * (p + 1) / 2), tim(p * (p + 1) / 2);
    std::vector<double> r64((size_t)8 * 2 * PP);
    for (int o = 0; o < 8; o++) {
        const double tx = (o & 1) ? 0.25 : -0.25, ty = (o & 2) ? 0.25 : -0.25, tz = (o & 4) ? 0.25 : -0.25;
        regular_tri<double>(p, tx, ty, tz, tre.data(), tim.data(), 1);
        double *dst = r64.data() + (size_t)o * 2 * PP;
        for (int n = 0; n < p; n++)
            for (int m = -n; m <= n; m++) {
                const int am = m < 0 ? -m : m;
                double re = tre[tri(n, am)], im = tim[tri(n, am)];
                if (m < 0) {
                    im = -im;
                    if (am & 1) {
                        re = -re;
                        im = -im;
                    }
                }
                dst[2 * full(n, m)] = re;
                dst[2 * full(n, m) + 1] = im;
            }
    }
    std::vector<float> r32(r64.size());
    for (size_t i = 0; i < r64.size(); i++) r32[i] = (float)r64[i];

    // M2M and L2L as real p^2 x p^2 maps of the packed expansions, one per child
    // octant o (the same sums as m2m_k and l2l_k, in FP64, applied to each unit
    // vector of the packed basis): column j = the map of e_j; stored [o][j][i].
    std::vector<float> mm((size_t)8 * PP * PP), ll((size_t)8 * PP * PP);
    std::vector<double> e(PP), out(PP);
    auto get = [&](int n, int m, double &re, double &im) {  // complex coefficient (n, m) of the packed e
        const int a = m < 0 ? -m : m;
        re = e[re_idx(n, a)];
        im = a ? e[im_idx(n, a)] : 0.0;
        if (m < 0) {
            im = -im;
            if (a & 1) {
                re = -re;
                im = -im;
            }
        }
    };
    for (int o = 0; o < 8; o++) {
        const double *R = r64.data() + (size_t)o * 2 * PP;
        for (int j0 = 0; j0 < PP; j0++) {
            std::fill(e.begin(), e.end(), 0.0);
            e[j0] = 1.0;
            // M2M: child (offset t_o from the parent centre, in parent widths) -> parent
            std::fill(out.begin(), out.end(), 0.0);
            for (int n = 0; n < p; n++)
                for (int m = 0; m <= n; m++) {
                    double sr = 0, si = 0;
                    for (int k = 0; k <= n; k++) {
                        const int j = n - k;
                        const double sc = std::ldexp(1.0, -j);
                        for (int l = -k; l <= k; l++) {
                            const int mu = m - l;
                            if (mu > j || mu < -j) continue;
                            const double rr = R[2 * full(k, l)], ri = -R[2 * full(k, l) + 1];
                            double mr, mi;
                            get(j, mu, mr, mi);
                            sr += sc * (rr * mr - ri * mi);
                            si += sc * (rr * mi + ri * mr);
                        }
                    }
                    out[re_idx(n, m)] = sr;
                    if (m) out[im_idx(n, m)] = si;
                }
            for (int i = 0; i < PP; i++) mm[((size_t)o * PP + j0) * PP + i] = (float)out[i];
            // L2L: parent -> child at offset t_o
            std::fill(out.begin(), out.end(), 0.0);
            for (int k = 0; k < p; k++)
                for (int l = 0; l <= k; l++) {
                    double sr = 0, si = 0;
                    for (int n = k; n < p; n++) {
                        const int d = n - k;
                        for (int m = -n; m <= n; m++) {
                            const int mu = m - l;
                            if (mu > d || mu < -d) continue;
                            double lr, li;
                            get(n, m, lr, li);
                            const double rr = R[2 * full(d, mu)], ri = -R[2 * full(d, mu) + 1];
                            sr += lr * rr - li * ri;
                            si += lr * ri + li * rr;
                        }
                    }
                    const double sc = std::ldexp(1.0, -(k + 1));
                    out[re_idx(k, l)] = sc * sr;
                    if (l) out[im_idx(k, l)] = sc * si;
                }
            for (int i = 0; i < PP; i++) ll[((size_t)o * PP + j0) * PP + i] = (float)out[i];
        }
    }
    h->m2m_mat.ensure(sizeof(float) * mm.size());
    h->l2l_mat.ensure(sizeof(float) * ll.size());
    FMM_CUDA_TRY(cudaMemcpy(h->m2m_mat.p, mm.data(), sizeof(float) * mm.size(), cudaMemcpyHostToDevice));
    FMM_CUDA_TRY(cudaMemcpy(h->l2l_mat.p, ll.data(), sizeof(float) * ll.size(), cudaMemcpyHostToDevice));
    h->rtab64.ensure(sizeof(double) * r64.size());
    h->rtab32.ensure(sizeof(float) * r32.size());
    FMM_CUDA_TRY(cudaMemcpy(h->rtab64.p, r64.data(), sizeof(double) * r64.size(), cudaMemcpyHostToDevice));
    FMM_CUDA_TRY(cudaMemcpy(h->rtab32.p, r32.data(), sizeof(float) * r32.size(), cudaMemcpyHostToDevice));
}

template <class T, class P4>
static void far_field_t(fmm_ctx *h, const P4 *xs, const T *rtab)
{
    cudaStream_t s = h->work;
    const int p = h->p, PP = p * p, ntri = p * (p + 1) / 2, Q = 2 * p - 1;
    const int nc = h->ncells;
    h->Mexp.ensure(sizeof(T) * (size_t)nc * PP);
    h->Lexp.ensure(sizeof(T) * (size_t)nc * PP);
    T *M = h->Mexp.as<T>(), *L = h->Lexp.as<T>();
    const Box *box = h->box.as<Box>();
    cudaEvent_t *ev = h->ev_cur;

    // P2M
    FMM_CUDA_TRY(cudaEventRecord(ev[2], s));
    bool p2m_done = false;
    if constexpr (std::is_same<T, float>::value) {
        if (h->nleaves > 0)
            p2m_done = p2m_warp_launch<P4>(p, h->nleaves, h->leaves.as<int>(), h->c_begin.as<int>(), h->c_end.as<int>(),
                                           h->c_xyz.as<int4>(), box, xs, M, s);
        if (p2m_done) {
            count_launch(h);
            check_launch("p2m");
        }
    }
    if (!p2m_done) {
        int chunk = std::min(64, (int)((48 * 1024) / (sizeof(T) * 2 * ntri)));
        chunk = std::max(chunk, 1);
        size_t smem = sizeof(T) * 2 * (size_t)ntri * chunk;
        p2m_k<T, P4><<<h->nleaves, 64, smem, s>>>(p, h->leaves.as<int>(), h->c_begin.as<int>(), h->c_end.as<int>(),
                                                  h->c_xyz.as<int4>(), box, xs, M, chunk);
        count_launch(h);
        check_launch("p2m");
    }
    // M2M, deepest level first
    FMM_CUDA_TRY(cudaEventRecord(ev[3], s));
    for (int l = h->depth - 1; l >= 0; l--) {
        const int ls = h->lvl_start[l], le = h->lvl_start[l + 1];
        const int64_t nt = (int64_t)(le - ls) * ntri;
        if (nt == 0) continue;
        if constexpr (std::is_same<T, float>::value)
            m2m_mv(PP, ls, le, h->c_child.as<int>(), h->c_nchild.as<int>(), h->c_xyz.as<int4>(), h->m2m_mat.as<float>(),
                   reinterpret_cast<float *>(M), s);
        else
            m2m_k<T><<<nblk(nt, 128), 128, 0, s>>>(p, ls, le, h->c_child.as<int>(), h->c_nchild.as<int>(),
                                                   h->c_xyz.as<int4>(), rtab, M);
        count_launch(h);
    }
    check_launch("m2m");
    // M2L
    FMM_CUDA_TRY(cudaEventRecord(ev[4], s));
    FMM_CUDA_TRY(cudaMemsetAsync(L, 0, sizeof(T) * (size_t)nc * PP, s));
    const int *st_off = stencil_offsets(h);
    if (h->depth >= 2) {
        if (std::is_same<T, float>::value && h->engine_used == FMM_M2L_TENSOR) {
            m2l_tensor(h, reinterpret_cast<float *>(L), reinterpret_cast<const float *>(M));
        } else if (h->engine_used == FMM_M2L_ROTATION) {
            m2l_rotation<T>(h, L, M);
        } else {
            const int tile = m2l_tile_size(h);
            size_t smem = sizeof(T) * 2 * ((size_t)Q * Q + (size_t)tile * PP) + sizeof(int) * 6 * tile;
            ensure_smem((const void *)m2l_cc_k<T>, smem);
            m2l_cc_k<T><<<h->ntiles_max, M2L_CC_T, smem, s>>>(
                p, h->m2l_tiles.as<M2LTile>(), reinterpret_cast<const int *>(h->m2l_misc.as<unsigned>() + 24 * (FMM_MAXLEVEL + 1)),
                h->m2l_tgt.as<int>(), h->c_xyz.as<int4>(), h->c_anchor.as<uint64_t>(), h->lvl_desc.as<LevelDesc>(),
                h->map_pool.as<int>(), h->st_dev.as<int4>(), st_off, M, L, tile);
            count_launch(h);
            check_launch("m2l");
        }
    }
    bool m2lx_done = false;
    if (h->n_m2lx > 0) {
        if constexpr (std::is_same<T, float>::value)
            m2lx_done = m2lx_f_launch(p, nc, h->m2lx_ptr.as<int>(), h->m2lx_src.as<int>(), h->c_xyz.as<int4>(),
                                      reinterpret_cast<const float *>(M), reinterpret_cast<float *>(L), s);
        if (m2lx_done) {
            count_launch(h);
            check_launch("m2l irregular");
        }
    }
    if (h->n_m2lx > 0 && !m2lx_done) {
        size_t smem = sizeof(T) * M2LX_W * 2 * ((size_t)Q * Q + PP) + sizeof(double) * M2LX_W * 2 * ntri;
        ensure_smem((const void *)m2lx_k<T>, smem);
        m2lx_k<T><<<nc, 32 * M2LX_W, smem, s>>>(p, nc, h->m2lx_ptr.as<int>(), h->m2lx_src.as<int>(), h->c_xyz.as<int4>(), M, L);
        count_launch(h);
        check_launch("m2l irregular");
    }
    // L2L, top down
    FMM_CUDA_TRY(cudaEventRecord(ev[5], s));
    for (int l = 0; l < h->depth; l++) {
        const int ls = h->lvl_start[l + 1], le = h->lvl_start[l + 2];
        const int64_t nt = (int64_t)(le - ls) * ntri;
        if (nt == 0) continue;
        if constexpr (std::is_same<T, float>::value)
            l2l_mv(PP, ls, le, h->c_parent.as<int>(), h->c_xyz.as<int4>(), h->l2l_mat.as<float>(),
                   reinterpret_cast<float *>(L), s);
        else
            l2l_k<T><<<nblk(nt, 128), 128, 0, s>>>(p, ls, le, h->c_parent.as<int>(), h->c_xyz.as<int4>(), rtab, L);
        count_launch(h);
    }
    check_launch("l2l");
    // L2P
    FMM_CUDA_TRY(cudaEventRecord(ev[6], s));
    h->far.ensure(sizeof(double4_32a) * (size_t)h->n);
    bool l2p_done = false;
    if constexpr (std::is_same<T, float>::value) {
        if (h->n > 0 && p >= 2 && p <= P2M_WARP_MAXP) {
            h->cgeo.ensure(sizeof(double4_32a) * (size_t)nc);
            cgeo_k<<<nblk(nc, 256), 256, 0, s>>>(nc, h->c_xyz.as<int4>(), box, h->cgeo.as<double4_32a>());
            count_launch(h);
            l2p_done = l2p_flat_launch<P4>(p, h->n, h->pcell.as<int>(), h->cgeo.as<double4_32a>(), xs,
                                           reinterpret_cast<const float *>(L), h->far.as<double4_32a>(), s);
        }
    }
    if (!l2p_done)
        l2p_k<T, P4><<<h->nleaves, 64, sizeof(T) * PP, s>>>(p, h->leaves.as<int>(), h->c_begin.as<int>(),
                                                            h->c_end.as<int>(), h->c_xyz.as<int4>(), box, xs, L,
                                                            h->far.as<double4_32a>());
    count_launch(h);
    check_launch("l2p");
    FMM_CUDA_TRY(cudaEventRecord(ev[7], s));
}


// ---------------------------------------------------------------------------
// Batched evaluation of many systems: the upward and downward passes as
// persistent kernels over a queue of per-warp work items (system, kind, cell,
// level), with per-system, per-level counters of finished cells. The items
// are queued in dependency order (P2M, then M2M from the deepest level up;
// L2L from the top level down, then L2P), so a warp waiting on a level only
// waits for items already taken by running warps. The arithmetic of every
// item is that of the single-system kernels.
// ---------------------------------------------------------------------------
constexpr long long BATCH_WAIT_CYCLES = 2000000000LL;  // about a second at 2 GHz

// wait until *cnt >= target (acquire); false, with bit 0 of *err set, once the
// wait has run for BATCH_WAIT_CYCLES or another wait of the launch gave up
__device__ bool batch_dep_wait(const unsigned *cnt, unsigned target, int *err)
{
    const long long t0 = clock64();
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
        if (v >= target) return true;
        if (*(volatile int *)err) return false;
        if (clock64() - t0 > BATCH_WAIT_CYCLES) {
            atomicOr(err, 1);
            return false;
        }
        __nanosleep(128);
    }
}

__device__ __forceinline__ void batch_done(unsigned *cnt)
{
    __threadfence();
    atomicAdd(cnt, 1u);
}

template <int P, int NR>
__global__ void __launch_bounds__(32 * MV_WARPS) batch_up_k(const BatchSys *__restrict__ sys, const int4 *__restrict__ items,
                                                           int nitems, int *__restrict__ queue,
                                                           const float *__restrict__ mat, int *__restrict__ err)
{
    __shared__ float sx[MV_WARPS][P * P];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(queue, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems) break;
        const int4 item = items[it];
        const BatchSys &S = sys[item.x];
        if (item.y == BATCH_P2M) {
            p2m_leaf_warp<P, float4>(item.z, lane, S.begin, S.end, S.xyz, S.box, S.xs, S.M);
        } else {
            // the children, one level down, are all final
            bool ok = true;
            if (lane == 0)
                ok = batch_dep_wait(S.cnt_up + item.w + 1, (unsigned)(S.lvl_start[item.w + 2] - S.lvl_start[item.w + 1]), err);
            if (!__shfl_sync(0xffffffffu, ok, 0)) continue;
            m2m_parent_warp<NR>(item.z, lane, P * P, S.child, S.nchild, S.xyz, mat, S.M, sx[w]);
        }
        __syncwarp();
        if (lane == 0) batch_done(S.cnt_up + item.w);
    }
}

template <int P, int NR>
__global__ void __launch_bounds__(32 * MV_WARPS) batch_down_k(const BatchSys *__restrict__ sys,
                                                             const int4 *__restrict__ items, int nitems,
                                                             int *__restrict__ queue, const float *__restrict__ mat,
                                                             int *__restrict__ err)
{
    __shared__ float sx[MV_WARPS][P * P];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(queue, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems) break;
        const int4 item = items[it];
        const BatchSys &S = sys[item.x];
        // L2L waits for the parents' level; L2P for its leaf's level
        const int lw = item.y == BATCH_L2L ? item.w - 1 : item.w;
        bool ok = true;
        if (lane == 0) ok = batch_dep_wait(S.cnt_dn + lw, (unsigned)(S.lvl_start[lw + 1] - S.lvl_start[lw]), err);
        if (!__shfl_sync(0xffffffffu, ok, 0)) continue;
        if (item.y == BATCH_L2L) {
            l2l_child_warp<NR>(item.z, lane, P * P, S.parent, S.xyz, mat, S.L, sx[w]);
            __syncwarp();
            if (lane == 0) batch_done(S.cnt_dn + item.w);
        } else {
            for (int j = S.begin[item.z] + lane; j < S.end[item.z]; j += 32)
                l2p_particle<P, float4, true>(j, item.z, S.cgeo, S.xs, S.L, S.far);
        }
    }
}

template <int P>
__global__ void __launch_bounds__(32 * M2LX_FW, 2) batch_m2lx_k(const BatchSys *__restrict__ sys,
                                                               const int2 *__restrict__ items, int nitems)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if ((int)blockIdx.x >= nitems) return;
    const int2 item = items[blockIdx.x];
    const BatchSys &S = sys[item.x];
    m2lx_f_cell<P>(item.y, S.m2lx_ptr, S.m2lx_src, S.xyz, S.M, S.L, smem_raw);
}

void batch_up(int p, int nsm, const BatchSys *sys, const int4 *items, int nitems, int *queue, const float *m2m_mat,
              int *err, cudaStream_t s)
{
    FMM_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(int), s));
    const unsigned g = (unsigned)nsm * 6;
    switch (p) {
#define FMM_BUP(PV) \
    case PV: batch_up_k<PV, (PV * PV + 31) / 32><<<g, 32 * MV_WARPS, 0, s>>>(sys, items, nitems, queue, m2m_mat, err); break;
        FMM_BUP(2) FMM_BUP(3) FMM_BUP(4) FMM_BUP(5) FMM_BUP(6) FMM_BUP(7) FMM_BUP(8) FMM_BUP(9) FMM_BUP(10)
#undef FMM_BUP
    default: throw Error{FMM_EINVAL, "batch: p must be in [2, 10]"};
    }
    check_launch("batch up");
}

void batch_down(int p, int nsm, const BatchSys *sys, const int4 *items, int nitems, int *queue, const float *l2l_mat,
                int *err, cudaStream_t s)
{
    FMM_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(int), s));
    const unsigned g = (unsigned)nsm * 6;
    switch (p) {
#define FMM_BDN(PV) \
    case PV: batch_down_k<PV, (PV * PV + 31) / 32><<<g, 32 * MV_WARPS, 0, s>>>(sys, items, nitems, queue, l2l_mat, err); break;
        FMM_BDN(2) FMM_BDN(3) FMM_BDN(4) FMM_BDN(5) FMM_BDN(6) FMM_BDN(7) FMM_BDN(8) FMM_BDN(9) FMM_BDN(10)
#undef FMM_BDN
    default: throw Error{FMM_EINVAL, "batch: p must be in [2, 10]"};
    }
    check_launch("batch down");
}

void batch_m2lx(int p, const BatchSys *sys, const int2 *items, int nitems, cudaStream_t s)
{
    if (nitems == 0) return;
    switch (p) {
#define FMM_BMX(PV)                                                                                       \
    case PV: {                                                                                            \
        constexpr size_t smem = m2lx_f_smem<PV>();                                                        \
        ensure_smem((const void *)batch_m2lx_k<PV>, smem);                                                \
        batch_m2lx_k<PV><<<nitems, 32 * M2LX_FW, smem, s>>>(sys, items, nitems);                          \
        break;                                                                                            \
    }
        FMM_BMX(2) FMM_BMX(3) FMM_BMX(4) FMM_BMX(5) FMM_BMX(6) FMM_BMX(7) FMM_BMX(8) FMM_BMX(9) FMM_BMX(10)
#undef FMM_BMX
    default: throw Error{FMM_EINVAL, "batch: p must be in [2, 10]"};
    }
    check_launch("batch m2l irregular");
}

void cell_geometry(fmm_ctx *h, cudaStream_t s)
{
    h->cgeo.ensure(sizeof(double4_32a) * (size_t)std::max(h->ncells, 1));
    cgeo_k<<<nblk(h->ncells, 256), 256, 0, s>>>(h->ncells, h->c_xyz.as<int4>(), h->box.as<Box>(), h->cgeo.as<double4_32a>());
    count_launch(h);
    check_launch("cell geometry");
}

void far_field(fmm_ctx *h)
{
    if (h->precision == FMM_FP64) {
        far_field_t<double, double4_32a>(h, h->xs64.as<double4_32a>(), h->rtab64.as<double>());
    } else if (h->dtype == FMM_F64) {
        far_field_t<float, double4_32a>(h, h->xs64.as<double4_32a>(), h->rtab32.as<float>());
    } else {
        far_field_t<float, float4>(h, h->xs32.as<float4>(), h->rtab32.as<float>());
    }
}

}  // namespace fmm
