// Near field (P2P), the FP64 direct sum and the final combine/unsort.
//
// P2P is the kernel that takes most of the FMM time (Sec. 3.1 of Yokota &
// Barba, arXiv:1106.2176) and the one their SIMD tuning targets (Sec. 3.2):
//   phi_i += sum_j q_j / r_ij,   grad_i -= sum_j q_j (x_i - x_j) / r_ij^3
// over the particles j of every leaf in the P2P list of i's leaf, skipping
// j == i and coincident pairs (r_ij = 0).
//
// GPU mapping: one block of 128 threads per target leaf. Each thread owns two
// targets (i and i + R, R = ceil(n_leaf / 2) rows) and one of S = 128 / R
// slices of the source stream, so a leaf of ~38 particles keeps ~114 of 128
// threads busy. Warp 0 plans each chunk of the concatenated source leaves (its
// pieces of runs); all threads copy it into shared memory as pair records
// while the previous chunk is computed. Threads of one slice read the same
// source pair (broadcast); the interaction runs on packed FP32 pairs (f32x2)
// and rsqrt on the CUDA cores. Block sums of up to ~128 source pairs, and the
// target leaf's own particles separately, are added with TwoSum into a
// per-thread (hi, lo) state; slices are combined with TwoSum in a fixed
// order, so the result does not depend on scheduling.
#include <algorithm>
#include <type_traits>

#include "fmm_internal.cuh"
#include "ptx_sm100.cuh"

namespace fmm {

static inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <class T>
struct Vec4;
template <>
struct Vec4<float> { using type = float4; };
template <>
struct Vec4<double> { using type = double4_32a; };

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

// One source s against target t. CHECK: the source segment may contain the
// target itself or particles at the same position (only the target's own
// leaf can: equal positions have equal Morton keys), which contribute nothing.
template <bool CHECK, class T, class T4>
__device__ __forceinline__ void interact(const T4 &t, const T4 &s, T &p, T &gx, T &gy, T &gz)
{
    const T dx = t.x - s.x, dy = t.y - s.y, dz = t.z - s.z;
    const T r2 = dx * dx + dy * dy + dz * dz;
    T ri = rsq(r2);
    if (CHECK) ri = r2 > T(0) ? ri : T(0);
    const T qr = s.w * ri;
    const T qr3 = qr * ri * ri;
    p += qr;
    gx -= qr3 * dx;
    gy -= qr3 * dy;
    gz -= qr3 * dz;
}

// The same with every coordinate carried as an FP32 pair (hi, lo): the
// difference (hi_i - hi_j) + (lo_i - lo_j) keeps the accuracy of FP64 inputs.
template <bool CHECK, class T4>
__device__ __forceinline__ void interact_ds(const T4 &t, const float4 &tl, const T4 &s, const float4 &sl, float &p,
                                            float &gx, float &gy, float &gz)
{
    const float dx = (t.x - s.x) + (tl.x - sl.x), dy = (t.y - s.y) + (tl.y - sl.y), dz = (t.z - s.z) + (tl.z - sl.z);
    const float r2 = dx * dx + dy * dy + dz * dz;
    float ri = rsqrtf(r2);
    if (CHECK) ri = r2 > 0.f ? ri : 0.f;
    const float qr = s.w * ri;
    const float qr3 = qr * ri * ri;
    p += qr;
    gx -= qr3 * dx;
    gy -= qr3 * dy;
    gz -= qr3 * dz;
}

// running sum (hi, lo) += b, error-free (TwoSum)
__device__ __forceinline__ void acc2(float &hi, float &lo, float b)
{
    const float s = hi + b;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (b - bb);
    hi = s;
    lo += err;
}
__device__ __forceinline__ void acc2(double &hi, double &lo, double b) { hi += b; }

#ifndef FMM_P2P_T
#define FMM_P2P_T 128
#endif
constexpr int P2P_T = FMM_P2P_T;  // threads per block (one target leaf)
// compile-time tuning knobs: targets per thread of the FP32 paths, and the
// minimum number of resident blocks per SM given to __launch_bounds__ (1
// leaves the register count to the compiler)
#ifndef FMM_P2P_TPT
#define FMM_P2P_TPT 2
#endif
#ifndef FMM_P2P_MINB
#define FMM_P2P_MINB 6
#endif
// sources per shared-memory chunk of the FP32-input path, and the number of
// chunk buffers (2: the next chunk is copied while the current one is
// computed; 3: the next two)
#ifndef FMM_P2P_CH
#define FMM_P2P_CH 688
#endif
// source segments (pieces of runs) per chunk of the packed path
constexpr int P2P_MAXSEG = 32;
#ifndef FMM_P2P_NBUF
#define FMM_P2P_NBUF 2
#endif
// source pairs summed in FP32 before they are folded into the TwoSum state,
// and the source pairs of one fully unrolled step of the pair loop
#ifndef FMM_P2P_FOLD
#define FMM_P2P_FOLD 256
#endif
#ifndef FMM_P2P_STEP
#define FMM_P2P_STEP 8
#endif

// One source against the TPT targets of a thread.
template <bool CHECK, bool DS, int TPT, class T, class T4>
__device__ __forceinline__ void p2p_one(const T4 &s, const float4 &q, const T4 (&x)[TPT], const float4 (&xl)[TPT],
                                        T (&b)[4 * TPT])
{
    if constexpr (DS) {
#pragma unroll
        for (int k = 0; k < TPT; k++) interact_ds<CHECK>(x[k], xl[k], s, q, b[4 * k], b[4 * k + 1], b[4 * k + 2], b[4 * k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < TPT; k++) interact<CHECK>(x[k], s, b[4 * k], b[4 * k + 1], b[4 * k + 2], b[4 * k + 3]);
    }
}

// Sources [j0, j1) of the shared chunk against the TPT targets of a thread:
// full blocks of 64 sources (fixed trip count, unrolled by 8) and a remainder;
// each block's sums are added to (h, lo) with TwoSum.
template <bool CHECK, bool DS, int TPT, class T, class T4>
__device__ __forceinline__ void p2p_range(int j0, int j1, const T4 *sh, const float4 *shlo, const T4 (&x)[TPT],
                                          const float4 (&xl)[TPT], T (&h)[4 * TPT], T (&lo)[4 * TPT])
{
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    int j = j0;
    for (; j + 64 <= j1; j += 64) {
        T b[4 * TPT];
#pragma unroll
        for (int c = 0; c < 4 * TPT; c++) b[c] = T(0);
#pragma unroll 8
        for (int jj = 0; jj < 64; jj++) p2p_one<CHECK, DS, TPT>(sh[j + jj], DS ? shlo[j + jj] : zero, x, xl, b);
#pragma unroll
        for (int c = 0; c < 4 * TPT; c++) acc2(h[c], lo[c], b[c]);
    }
    if (j < j1) {
        T b[4 * TPT];
#pragma unroll
        for (int c = 0; c < 4 * TPT; c++) b[c] = T(0);
#pragma unroll 4
        for (; j < j1; j++) p2p_one<CHECK, DS, TPT>(sh[j], DS ? shlo[j] : zero, x, xl, b);
#pragma unroll
        for (int c = 0; c < 4 * TPT; c++) acc2(h[c], lo[c], b[c]);
    }
}

// ---------------------------------------------------------------------------
// Packed FP32 pairs (sm_100 and later: add/sub/mul/fma .f32x2). Two sources
// are handled per instruction against one target; the shared chunk holds the
// sources as pair records (x0 x1 y0 y1 | z0 z1 q0 q1), so one 16-byte load
// gives two packed operands. Each packed instruction does the work of two
// FP32 ones in one issue slot.
// ---------------------------------------------------------------------------
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2_pack(float lo, float hi)
{
    f2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void f2_unpack(f2 a, float &lo, float &hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a)); }

// Two sources (packed sx..sq) against one target (tx, ty, tz duplicated in
// both halves): p += q / r, g += q (x_j - x_i) / r^3, per half.
template <bool CHECK>
__device__ __forceinline__ void interact_pk(f2 sx, f2 sy, f2 sz, f2 sq, f2 tx, f2 ty, f2 tz, f2 &p, f2 &gx, f2 &gy,
                                            f2 &gz)
{
    const f2 dx = f2_sub(sx, tx), dy = f2_sub(sy, ty), dz = f2_sub(sz, tz);
    const f2 r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
    float a, b;
    f2_unpack(r2, a, b);
    float ra = rsqrtf(a), rb = rsqrtf(b);
    if (CHECK) {
        ra = a > 0.f ? ra : 0.f;
        rb = b > 0.f ? rb : 0.f;
    }
    const f2 ri = f2_pack(ra, rb);
    const f2 qr = f2_mul(sq, ri);
    p = f2_add(p, qr);
    const f2 qr3 = f2_mul(qr, f2_mul(ri, ri));
    gx = f2_fma(qr3, dx, gx);
    gy = f2_fma(qr3, dy, gy);
    gz = f2_fma(qr3, dz, gz);
}

// Sources [j0, j1) of a pair-record chunk against the TPT targets of a
// thread, added into the packed block sums acc (the two halves hold even and
// odd sources). An odd source at either end is taken alone and added to the
// low half; the pairs between run in fully unrolled steps and a tail.
// `cnt` counts the pairs in acc since the last fold.
template <bool CHECK, int TPT>
__device__ __forceinline__ void p2p_range_pk(int j0, int j1, const float *shf, const f2 (&tx)[TPT], const f2 (&ty)[TPT],
                                             const f2 (&tz)[TPT], f2 (&acc)[4 * TPT], int &cnt)
{
    auto single = [&](int j) {
        const float *r = shf + 8 * (j >> 1) + (j & 1);
        const float4 sj = make_float4(r[0], r[2], r[4], r[6]);
#pragma unroll
        for (int k = 0; k < TPT; k++) {
            float xi, yi, zi, u;
            f2_unpack(tx[k], xi, u);
            f2_unpack(ty[k], yi, u);
            f2_unpack(tz[k], zi, u);
            float pp = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
            interact<CHECK>(make_float4(xi, yi, zi, 0.f), sj, pp, gx, gy, gz);
            // interact() and the packed sums both hold q (x_j - x_i) / r^3
            acc[4 * k] = f2_add(acc[4 * k], f2_pack(pp, 0.f));
            acc[4 * k + 1] = f2_add(acc[4 * k + 1], f2_pack(gx, 0.f));
            acc[4 * k + 2] = f2_add(acc[4 * k + 2], f2_pack(gy, 0.f));
            acc[4 * k + 3] = f2_add(acc[4 * k + 3], f2_pack(gz, 0.f));
        }
        cnt++;
    };
    int a = j0, b = j1;
    if (a < b && (a & 1)) single(a++);
    if (a < b && (b & 1)) single(--b);
    const ulonglong2 *pr = reinterpret_cast<const ulonglong2 *>(shf);
    int k = a >> 1;
    const int k1 = b >> 1;
    cnt += k1 - k;
    for (; k + FMM_P2P_STEP <= k1; k += FMM_P2P_STEP) {
#pragma unroll
        for (int kk = 0; kk < FMM_P2P_STEP; kk++) {
            const ulonglong2 A = pr[2 * (k + kk)], B = pr[2 * (k + kk) + 1];
#pragma unroll
            for (int t = 0; t < TPT; t++)
                interact_pk<CHECK>(A.x, A.y, B.x, B.y, tx[t], ty[t], tz[t], acc[4 * t], acc[4 * t + 1], acc[4 * t + 2],
                                   acc[4 * t + 3]);
        }
    }
    for (; k < k1; k++) {
        const ulonglong2 A = pr[2 * k], B = pr[2 * k + 1];
#pragma unroll
        for (int t = 0; t < TPT; t++)
            interact_pk<CHECK>(A.x, A.y, B.x, B.y, tx[t], ty[t], tz[t], acc[4 * t], acc[4 * t + 1], acc[4 * t + 2],
                               acc[4 * t + 3]);
    }
}

// the packed block sums are added, half by half, into the thread's (hi, lo)
// state with TwoSum (hl[c * P2P_T], hl[(4 TPT + c) * P2P_T] in shared memory)
template <int TPT>
__device__ __forceinline__ void p2p_fold_pk(f2 (&acc)[4 * TPT], float *hl)
{
#pragma unroll
    for (int c = 0; c < 4 * TPT; c++) {
        float u, v;
        f2_unpack(acc[c], u, v);
        acc2(hl[c * P2P_T], hl[(4 * TPT + c) * P2P_T], u + v);
        acc[c] = 0ull;
    }
}

__device__ __forceinline__ void cpa4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cpa16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Where the source stream of a target leaf stands (block-uniform).
struct RunCursor {
    int k, k1, off;
};

// One block per target leaf. A thread owns TPT targets (rows of R =
// ceil(n / TPT)) and one of S = 128 / R slices of the source stream. Sources
// come as particle runs (adjacent source leaves merged); chunks of CH sources
// are copied into shared memory with cp.async, the next chunk while the
// current one is computed (two buffers). Only the target leaf's own particles
// need the j == i / r == 0 test. Slices are reduced in a fixed order.
// DS: FP32 (hi, lo) coordinates for FP64 inputs.
template <class T, bool DS, int TPT>
__global__ void __launch_bounds__(P2P_T, sizeof(T) == 4 ? FMM_P2P_MINB : 1) p2p_k(const typename Vec4<T>::type *__restrict__ xs, const float4 *__restrict__ xlo,
                                               const int *__restrict__ leaves, const int *__restrict__ begin,
                                               const int *__restrict__ end, const int *__restrict__ ptr,
                                               const int2 *__restrict__ runs, const int *__restrict__ nrun,
                                               double4_32a *__restrict__ near)
{
    using T4 = typename Vec4<T>::type;
    constexpr bool PK = std::is_same<T, float>::value && !DS;  // packed pairs (pair-record chunks)
    constexpr int CH = DS ? 512 : (sizeof(T) == 8 ? 512 : FMM_P2P_CH);
    constexpr int NB = PK ? FMM_P2P_NBUF : 2;
    static_assert(NB == 2 || NB == 3, "two or three chunk buffers");
    static_assert(!(PK && NB == 3), "the packed path plans one chunk ahead");
    __shared__ T4 sh[NB][CH];
    __shared__ float4 shlo[DS ? 2 : 1][DS ? CH : 1];
    __shared__ float hls[PK ? 8 * TPT * P2P_T : 1];  // packed path: per-thread TwoSum state, column-major
    // packed path: per chunk, its source segments (first source, count,
    // position in the chunk) and (segments, fill, own-leaf range), planned by
    // warp 0; three tables rotate so none is rewritten while it is read
    __shared__ int4 tseg[PK ? 3 : 1][PK ? P2P_MAXSEG : 1];
    __shared__ int4 tinf[PK ? 3 : 1];
    static_assert(sizeof(T4) * NB * CH >= sizeof(double) * P2P_T * 4 * TPT, "slice sums reuse the source buffers");
    double *red = reinterpret_cast<double *>(&sh[0][0]);  // slice sums, after the last chunk
    const int A = leaves[blockIdx.x];
    const int tb = begin[A], te = end[A];
    const int r0 = ptr[A], r1 = ptr[A] + nrun[A];

    // copy the next chunk into buffer bf; returns its length and where the
    // target leaf's own particles sit in it ([slo, shi), empty if absent)
    auto stage = [&](RunCursor &cur, int bf, int &slo, int &shi) -> int {
        int fill = 0;
        slo = shi = 0;
        while (cur.k < cur.k1 && fill < CH) {
            const int2 rr = runs[cur.k];
            const int g0 = rr.x + cur.off;
            const int len = rr.y - g0;
            const int take = min(len, CH - fill);
            for (int j = threadIdx.x; j < take; j += P2P_T) {
                if constexpr (PK) {  // source c -> pair record c / 2, half c % 2
                    const int c = fill + j;
                    float *d = reinterpret_cast<float *>(&sh[bf][0]) + 8 * (c >> 1) + (c & 1);
                    const float *g = reinterpret_cast<const float *>(xs + g0 + j);
                    cpa4(d, g);
                    cpa4(d + 2, g + 1);
                    cpa4(d + 4, g + 2);
                    cpa4(d + 6, g + 3);
                } else {
#pragma unroll
                    for (int c = 0; c < (int)(sizeof(T4) / 16); c++)  // 16-byte pieces of one particle
                        cpa16(reinterpret_cast<char *>(&sh[bf][fill + j]) + 16 * c,
                              reinterpret_cast<const char *>(xs + g0 + j) + 16 * c);
                    if constexpr (DS) cpa16(&shlo[bf][fill + j], xlo + g0 + j);
                }
            }
            const int a = max(g0, tb), b = min(g0 + take, te);
            if (a < b) {
                slo = fill + a - g0;
                shi = fill + b - g0;
            }
            fill += take;
            if (take == len) {
                cur.k++;
                cur.off = 0;
            } else cur.off += take;
        }
        cpa_commit();
        return fill;
    };

    // warp 0: the next chunk's segments from the run cursor, 32 runs per step
    // (a warp scan of their lengths gives their positions in the chunk)
    auto plan = [&](RunCursor &cur, int tb_) {
        const int lane = threadIdx.x & 31;
        int fill = 0, nseg = 0;
        if (lane == 0) tinf[tb_] = make_int4(0, 0, 0, 0);
        __syncwarp();
        while (cur.k < cur.k1 && fill < CH && nseg < P2P_MAXSEG) {
            const int k = cur.k + lane;
            int g0 = 0, len = 0;
            if (k < cur.k1) {
                const int2 rr = runs[k];
                g0 = rr.x + (lane == 0 ? cur.off : 0);
                len = rr.y - g0;
            }
            int incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int start = fill + incl - len;
            int take = max(0, min(len, CH - start));
            if (nseg + lane >= P2P_MAXSEG) take = 0;
            const int cnt = __popc(__ballot_sync(0xffffffffu, take > 0));
            if (cnt == 0) break;
            if (take > 0) {
                tseg[tb_][nseg + lane] = make_int4(g0, take, start, 0);
                const int a = max(g0, tb), b = min(g0 + take, te);
                if (a < b) {
                    tinf[tb_].z = start + a - g0;
                    tinf[tb_].w = start + b - g0;
                }
            }
            const int lt = __shfl_sync(0xffffffffu, take, cnt - 1), ll = __shfl_sync(0xffffffffu, len, cnt - 1),
                      ls = __shfl_sync(0xffffffffu, start, cnt - 1);
            fill = ls + lt;
            nseg += cnt;
            if (lt == ll) {
                cur.k += cnt;
                cur.off = 0;
            } else {
                cur.off = (cnt == 1 ? cur.off : 0) + lt;
                cur.k += cnt - 1;
            }
        }
        __syncwarp();
        if (lane == 0) {
            tinf[tb_].x = nseg;
            tinf[tb_].y = fill;
        }
    };
    // every thread: copy its sources of the planned chunk into buffer bf
    auto stage_planned = [&](int tb_, int bf) {
        const int ns = tinf[tb_].x;
        float *base = reinterpret_cast<float *>(&sh[bf][0]);
        for (int sgi = 0; sgi < ns; sgi++) {
            const int4 e = tseg[tb_][sgi];
            for (int j = threadIdx.x; j < e.y; j += P2P_T) {  // source c -> pair record c / 2, half c % 2
                const int c = e.z + j;
                float *d = base + 8 * (c >> 1) + (c & 1);
                const float *g = reinterpret_cast<const float *>(xs + e.x + j);
                cpa4(d, g);
                cpa4(d + 2, g + 1);
                cpa4(d + 4, g + 2);
                cpa4(d + 6, g + 3);
            }
        }
        cpa_commit();
    };

    for (int t0 = tb; t0 < te; t0 += TPT * P2P_T) {
        const int nt = min(TPT * P2P_T, te - t0);
        const int R = (nt + TPT - 1) / TPT;
        const int S = max(1, P2P_T / R);
        const int row = threadIdx.x % R, sl = threadIdx.x / R;
        const bool act = sl < S;
        T4 x[TPT];
        float4 xl[TPT];
#pragma unroll
        for (int k = 0; k < TPT; k++) {
            const int i = (act && row + k * R < nt) ? t0 + row + k * R : t0;
            x[k] = xs[i];
            if constexpr (DS) xl[k] = xlo[i];
            else xl[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        f2 tx[TPT], ty[TPT], tz[TPT];
#pragma unroll
        for (int k = 0; k < TPT; k++) {
            if constexpr (PK) {
                tx[k] = f2_pack((float)x[k].x, (float)x[k].x);
                ty[k] = f2_pack((float)x[k].y, (float)x[k].y);
                tz[k] = f2_pack((float)x[k].z, (float)x[k].z);
            } else tx[k] = ty[k] = tz[k] = 0ull;
        }
        T h[4 * TPT], lo[4 * TPT];
#pragma unroll
        for (int c = 0; c < 4 * TPT; c++) h[c] = lo[c] = T(0);
        f2 pacc[4 * TPT];  // packed path: block sums of the current fold
        int pcnt = 0;
#pragma unroll
        for (int c = 0; c < 4 * TPT; c++) pacc[c] = 0ull;
        if constexpr (PK) {
#pragma unroll
            for (int c = 0; c < 8 * TPT; c++) hls[c * P2P_T + threadIdx.x] = 0.f;
        }
        RunCursor cur{r0, r1, 0};
        __syncthreads();  // buffers free (previous target block or slice sums)
        int slo = 0, shi = 0, fill = 0, ti = 0;  // ti: table of the current chunk
        if constexpr (PK) {
            if (threadIdx.x < 32) plan(cur, 0);
            __syncthreads();
            const int4 inf = tinf[0];
            fill = inf.y;
            slo = inf.z;
            shi = inf.w;
            if (fill > 0) stage_planned(0, 0);
        } else {
            fill = stage(cur, 0, slo, shi);
        }
        int bf = 0;
        // NB = 3: chunk i + 1 is staged ahead as well; chunk i + 2 goes into
        // the buffer of chunk i - 1 once every thread has passed the barrier
        // that follows chunk i - 1
        int nslo = 0, nshi = 0, nfill = 0;
        if (NB == 3 && cur.k < cur.k1) nfill = stage(cur, 1, nslo, nshi);
        while (fill > 0) {
            int n2lo = 0, n2hi = 0, n2fill = 0;
            if constexpr (NB == 3) {
                if (nfill > 0) cpa_wait1();
                else cpa_wait0();
                __syncthreads();  // chunk bf complete; chunk bf - 1 consumed by every thread
                if (cur.k < cur.k1) n2fill = stage(cur, bf == 0 ? 2 : bf - 1, n2lo, n2hi);
            } else if constexpr (PK) {
                // warp 0 plans chunk bf + 1; after the barrier chunk bf is
                // complete, every thread has finished chunk bf - 1, and all copy
                // chunk bf + 1 into its buffer while chunk bf is computed
                cpa_wait0();
                const int tn = ti == 2 ? 0 : ti + 1;
                if (threadIdx.x < 32) plan(cur, tn);
                __syncthreads();
                const int4 inf = tinf[tn];
                nfill = inf.y;
                nslo = inf.z;
                nshi = inf.w;
                if (nfill > 0) stage_planned(tn, bf ^ 1);
                ti = tn;
            } else {
                // one barrier per chunk: after it, chunk bf is complete and
                // every thread has finished chunk bf - 1, whose buffer then
                // takes chunk bf + 1 while chunk bf is computed
                cpa_wait0();
                __syncthreads();
                nfill = cur.k < cur.k1 ? stage(cur, bf ^ 1, nslo, nshi) : 0;
            }
            if (act) {
                if constexpr (PK) {
                    // slice bounds on even sources, so only the target leaf's
                    // own segment and an odd chunk end leave single sources
                    const int np = (fill + 1) >> 1;  // np * S <= (CH / 2) * P2P_T fits in 32 bits
                    const int jlo = min(fill, 2 * ((np * sl) / S));
                    const int jhi = min(fill, 2 * ((np * (sl + 1)) / S));
                    const float *sb = reinterpret_cast<const float *>(&sh[bf][0]);
                    // the target leaf's own particles (the nearest, largest
                    // terms) are summed and folded on their own
                    const bool own = max(jlo, slo) < min(jhi, shi);
                    p2p_range_pk<false, TPT>(jlo, min(jhi, slo), sb, tx, ty, tz, pacc, pcnt);
                    if (own) {
                        p2p_fold_pk<TPT>(pacc, hls + threadIdx.x);
                        p2p_range_pk<true, TPT>(max(jlo, slo), min(jhi, shi), sb, tx, ty, tz, pacc, pcnt);
                        p2p_fold_pk<TPT>(pacc, hls + threadIdx.x);
                        pcnt = 0;
                    }
                    p2p_range_pk<false, TPT>(max(jlo, shi), jhi, sb, tx, ty, tz, pacc, pcnt);
                    if (pcnt >= FMM_P2P_FOLD) {
                        p2p_fold_pk<TPT>(pacc, hls + threadIdx.x);
                        pcnt = 0;
                    }
                } else {
                    const int jlo = (int)(((long long)fill * sl) / S), jhi = (int)(((long long)fill * (sl + 1)) / S);
                    const T4 *sb = sh[bf];
                    const float4 *sbl = shlo[DS ? bf : 0];
                    p2p_range<false, DS, TPT>(jlo, min(jhi, slo), sb, sbl, x, xl, h, lo);
                    p2p_range<true, DS, TPT>(max(jlo, slo), min(jhi, shi), sb, sbl, x, xl, h, lo);
                    p2p_range<false, DS, TPT>(max(jlo, shi), jhi, sb, sbl, x, xl, h, lo);
                }
            }
            if constexpr (NB == 3) {
                bf = bf == 2 ? 0 : bf + 1;
                fill = nfill;
                slo = nslo;
                shi = nshi;
                nfill = n2fill;
                nslo = n2lo;
                nshi = n2hi;
            } else {
                bf ^= 1;
                fill = nfill;
                slo = nslo;
                shi = nshi;
            }
        }
        __syncthreads();  // the last chunk consumed before the slice sums reuse it
        if (act) {
            if constexpr (PK) {
                p2p_fold_pk<TPT>(pacc, hls + threadIdx.x);
#pragma unroll
                for (int c = 0; c < 4 * TPT; c++) {
                    h[c] = hls[c * P2P_T + threadIdx.x];
                    lo[c] = hls[(4 * TPT + c) * P2P_T + threadIdx.x];
                }
            }
            if constexpr (sizeof(T) == 4) {
                float2 *red2 = reinterpret_cast<float2 *>(red);
#pragma unroll
                for (int c = 0; c < 4 * TPT; c++) red2[(sl * R + row) * 4 * TPT + c] = make_float2(h[c], lo[c]);
            } else {
#pragma unroll
                for (int c = 0; c < 4 * TPT; c++) red[(sl * R + row) * 4 * TPT + c] = (double)h[c] + (double)lo[c];
            }
        }
        __syncthreads();
        if ((int)threadIdx.x < R) {
            double o[4 * TPT];
            if constexpr (sizeof(T) == 4) {
                // slices in fixed order, compensated in FP32 (TwoSum of the
                // leading parts, the trailing parts added), one conversion each
                const float2 *red2 = reinterpret_cast<const float2 *>(red);
                float oh[4 * TPT], ol[4 * TPT];
#pragma unroll
                for (int c = 0; c < 4 * TPT; c++) oh[c] = ol[c] = 0.f;
                for (int s2 = 0; s2 < S; s2++)
#pragma unroll
                    for (int c = 0; c < 4 * TPT; c++) {
                        const float2 v = red2[(s2 * R + threadIdx.x) * 4 * TPT + c];
                        acc2(oh[c], ol[c], v.x);
                        ol[c] += v.y;
                    }
#pragma unroll
                for (int c = 0; c < 4 * TPT; c++) o[c] = (double)oh[c] + (double)ol[c];
            } else {
#pragma unroll
                for (int c = 0; c < 4 * TPT; c++) o[c] = 0.0;
                for (int s2 = 0; s2 < S; s2++)
#pragma unroll
                    for (int c = 0; c < 4 * TPT; c++) o[c] += red[(s2 * R + threadIdx.x) * 4 * TPT + c];
            }
#pragma unroll
            for (int kk = 0; kk < TPT; kk++)
                if ((int)threadIdx.x + kk * R < nt)
                    near[t0 + threadIdx.x + kk * R] = make_double4_32a(o[4 * kk], o[4 * kk + 1], o[4 * kk + 2], o[4 * kk + 3]);
        }
    }
}


// ---------------------------------------------------------------------------
// Packed P2P of FP32 inputs with source chunks staged by bulk copies.
//
// The sorted particles are kept a second time as pair records
// (x0 x1 y0 y1 | z0 z1 q0 q1), each leaf padded to an even count by a
// zero-charge copy of its last particle, so every run of source leaves is a
// whole number of records and copies as one contiguous block. Warp 0 turns
// the target leaf's runs into chunks of up to PR_CHP records: one
// cp.async.bulk per run piece, completion counted in bytes on the chunk's
// mbarrier, PR_D chunks ahead of the one being computed. The warps compute a
// chunk as soon as it has landed and release it with one arrival each, so no
// CTA-wide barrier separates the chunks. The arithmetic and the summation
// order per thread are those of p2p_k. Ring shape (2 buffers of 344 pairs,
// one chunk ahead, packed sums folded every 256 pairs) from a sweep at
// N = 10^7: 31.5 ms against 32.3 ms for the cp.async staging of p2p_k.
// ---------------------------------------------------------------------------
#ifndef FMM_PR_NB
#define FMM_PR_NB 2
#endif
#ifndef FMM_PR_CHP
#define FMM_PR_CHP 344
#endif
#ifndef FMM_PR_D
#define FMM_PR_D (FMM_PR_NB - 1)
#endif
constexpr int PR_NB = FMM_PR_NB;    // chunk buffers
constexpr int PR_CHP = FMM_PR_CHP;  // source pairs per chunk
constexpr int PR_D = FMM_PR_D;      // chunk c + PR_D is produced when chunk c starts (PR_D < PR_NB)
static_assert(PR_D >= 1 && PR_D < PR_NB, "produce ahead within the ring");

// flag[i] = 1 for the last particle of a leaf with an odd count
__global__ void pr_flag_k(int64_t n, const int *__restrict__ pcell, const int *__restrict__ begin,
                          const int *__restrict__ end, unsigned *__restrict__ flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = pcell[i];
    flag[i] = (i == end[c] - 1 && ((end[c] - begin[c]) & 1)) ? 1u : 0u;
}

// particle i sits at padded position i + pad[i] (half (i + pad[i]) & 1 of
// record (i + pad[i]) / 2); the last particle of an odd leaf, at an even
// position, also fills the other half with its position and charge zero
__global__ void pr_fill_k(int64_t n, const float4 *__restrict__ xs, const unsigned *__restrict__ pad,
                          const unsigned *__restrict__ flag, float *__restrict__ pairs)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = xs[i];
    const int64_t pi = i + pad[i];
    float *rec = pairs + 8 * (pi >> 1);
    const int hh = (int)(pi & 1);
    rec[hh] = a.x;
    rec[2 + hh] = a.y;
    rec[4 + hh] = a.z;
    rec[6 + hh] = a.w;
    if (flag[i]) {
        rec[1] = a.x;
        rec[3] = a.y;
        rec[5] = a.z;
        rec[7] = 0.f;
    }
}

// runs of particles [b, e) (whole leaves) -> runs of records
// [(b + pad[b]) / 2, (e + pad[e - 1] + flag[e - 1]) / 2)
__global__ void pr_runs_k(int nleaves, const int *__restrict__ leaves, const int *__restrict__ ptr,
                          const int *__restrict__ nrun, const int2 *__restrict__ runs, const unsigned *__restrict__ pad,
                          const unsigned *__restrict__ flag, int2 *__restrict__ runs_pr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaves) return;
    const int A = leaves[i];
    for (int k = ptr[A]; k < ptr[A] + nrun[A]; k++) {
        const int2 r = runs[k];
        runs_pr[k] = make_int2((int)((r.x + pad[r.x]) >> 1), (int)((r.y + pad[r.y - 1] + flag[r.y - 1]) >> 1));
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t tx)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(tx) : "memory");
}

// pairs [k0, k1) of a chunk against the TPT targets of a thread (every pair whole)
template <bool CHECK, int TPT>
__device__ __forceinline__ void p2p_pairs_pk(int k, int k1, const ulonglong2 *pr, const f2 (&tx)[TPT], const f2 (&ty)[TPT],
                                             const f2 (&tz)[TPT], f2 (&acc)[4 * TPT], int &cnt)
{
    cnt += max(0, k1 - k);
    for (; k + FMM_P2P_STEP <= k1; k += FMM_P2P_STEP) {
#pragma unroll
        for (int kk = 0; kk < FMM_P2P_STEP; kk++) {
            const ulonglong2 A = pr[2 * (k + kk)], B = pr[2 * (k + kk) + 1];
#pragma unroll
            for (int t = 0; t < TPT; t++)
                interact_pk<CHECK>(A.x, A.y, B.x, B.y, tx[t], ty[t], tz[t], acc[4 * t], acc[4 * t + 1], acc[4 * t + 2],
                                   acc[4 * t + 3]);
        }
    }
    for (; k < k1; k++) {
        const ulonglong2 A = pr[2 * k], B = pr[2 * k + 1];
#pragma unroll
        for (int t = 0; t < TPT; t++)
            interact_pk<CHECK>(A.x, A.y, B.x, B.y, tx[t], ty[t], tz[t], acc[4 * t], acc[4 * t + 1], acc[4 * t + 2],
                               acc[4 * t + 3]);
    }
}

// shared memory of one P2P block: chunk ring, TwoSum state, chunk table, barriers
template <int TPT>
struct PRShared {
    __align__(128) float4 buf[PR_NB][2 * PR_CHP];  // pair records, two float4 each
    float hls[8 * TPT * P2P_T];                    // per-thread TwoSum state, column-major
    int4 info[PR_NB];                              // per chunk: records, own-leaf records [lo, hi)
    uint64_t full[PR_NB], empty[PR_NB];
    int item;                                      // persistent blocks: the current work item
};

template <int TPT>
__device__ __forceinline__ void p2p_pr_init(PRShared<TPT> &sh)
{
    if (threadIdx.x == 0) {
        for (int b = 0; b < PR_NB; b++) {
            mbar_init(&sh.full[b], 1);
            mbar_init(&sh.empty[b], P2P_T / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// near field of target leaf A; cc counts the chunks this block has consumed
// (it carries the barrier phases from one leaf to the next)
template <int TPT>
__device__ __forceinline__ void p2p_pr_leaf(int A, int &cc, PRShared<TPT> &sh, const float4 *__restrict__ xs,
                                            const float *__restrict__ pairs, const unsigned *__restrict__ pad,
                                            const unsigned *__restrict__ flag, const int *__restrict__ begin,
                                            const int *__restrict__ end, const int *__restrict__ ptr,
                                            const int2 *__restrict__ runs_pr, const int *__restrict__ nrun,
                                            double4_32a *__restrict__ near, int *__restrict__ err)
{
    auto &buf = sh.buf;
    float *hls = sh.hls;
    int4 *info = sh.info;
    uint64_t *full = sh.full, *empty = sh.empty;
    static_assert(sizeof(sh.buf) >= sizeof(float2) * P2P_T * 4 * TPT, "slice sums reuse the chunk buffers");
    float2 *red2 = reinterpret_cast<float2 *>(&buf[0][0]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tb = begin[A], te = end[A];
    const int k0 = ptr[A], k1 = ptr[A] + nrun[A];
    const int op0 = (int)((tb + pad[tb]) >> 1), op1 = (int)((te + pad[te - 1] + flag[te - 1]) >> 1);
    bool bad = false;  // a bounded wait ran out: results of this leaf are void, err is set

    for (int t0 = tb; t0 < te; t0 += TPT * P2P_T) {
        const int nt = min(TPT * P2P_T, te - t0);
        const int R = (nt + TPT - 1) / TPT;
        const int S = max(1, P2P_T / R);
        const int row = threadIdx.x % R, sl = threadIdx.x / R;
        const bool act = sl < S;
        f2 tx[TPT], ty[TPT], tz[TPT];
#pragma unroll
        for (int k = 0; k < TPT; k++) {
            const int i = (act && row + k * R < nt) ? t0 + row + k * R : t0;
            const float4 x = xs[i];
            tx[k] = f2_pack(x.x, x.x);
            ty[k] = f2_pack(x.y, x.y);
            tz[k] = f2_pack(x.z, x.z);
        }
        f2 pacc[4 * TPT];
        int pcnt = 0;
#pragma unroll
        for (int c = 0; c < 4 * TPT; c++) pacc[c] = 0ull;
#pragma unroll
        for (int c = 0; c < 8 * TPT; c++) hls[c * P2P_T + threadIdx.x] = 0.f;

        // producer state (warp 0): run cursor in records, next chunk to make
        int ck = k0, coff = 0, pnext = cc;
        bool pdone = false;
        // warp 0: chunk c into buffer c % PR_NB once its previous chunk is
        // released; a chunk with no records marks the end of the stream
        auto produce = [&](int c) {
            const int b = c % PR_NB;
            bool ok = true;
            if (c >= PR_NB) ok = mbar_wait(&empty[b], (uint32_t)(((c - PR_NB) / PR_NB) & 1));
            if (!__all_sync(0xffffffffu, ok)) {
                bad = true;
                if (lane == 0) atomicExch(err, 1);
            }
            int fill = 0, slo = 0, shi = 0;
            while (!bad && ck < k1 && fill < PR_CHP) {
                const int k = ck + lane;
                int g0 = 0, len = 0;
                if (k < k1) {
                    const int2 rr = runs_pr[k];
                    g0 = rr.x + (lane == 0 ? coff : 0);
                    len = rr.y - g0;
                }
                int incl = len;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int start = fill + incl - len;
                const int take = max(0, min(len, PR_CHP - start));
                const int cnt = __popc(__ballot_sync(0xffffffffu, take > 0));
                if (cnt == 0) break;
                int a0 = 0, a1 = 0;
                if (take > 0) {
                    mbar_expect_tx(&full[b], (uint32_t)take * 32u);
                    bulk_g2s(smem_u32(&buf[b][2 * start]), pairs + 8 * (size_t)g0, (uint32_t)take * 32u, &full[b]);
                    a0 = max(g0, op0);
                    a1 = min(g0 + take, op1);
                }
                // the target leaf is one leaf of one run: at most one lane holds it
                const unsigned own = __ballot_sync(0xffffffffu, a0 < a1);
                if (own) {
                    const int src = __ffs(own) - 1;
                    slo = __shfl_sync(0xffffffffu, start + a0 - g0, src);
                    shi = __shfl_sync(0xffffffffu, start + a1 - g0, src);
                }
                const int lt = __shfl_sync(0xffffffffu, take, cnt - 1), ll = __shfl_sync(0xffffffffu, len, cnt - 1),
                          ls = __shfl_sync(0xffffffffu, start, cnt - 1);
                fill = ls + lt;
                if (lt == ll) {
                    ck += cnt;
                    coff = 0;
                } else {
                    coff = (cnt == 1 ? coff : 0) + lt;
                    ck += cnt - 1;
                }
            }
            __syncwarp();
            if (lane == 0) {
                info[b] = make_int4(fill, slo, shi, 0);
                mbar_arrive(&full[b]);
            }
            __syncwarp();
            return fill;
        };
        auto produce_upto = [&](int last) {
            while (!pdone && pnext <= last) {
                if (produce(pnext) == 0) pdone = true;
                pnext++;
            }
        };
        if (warp == 0) produce_upto(cc + PR_D);

        for (;;) {
            if (warp == 0) produce_upto(cc + PR_D);
            const int b = cc % PR_NB;
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[b], (uint32_t)((cc / PR_NB) & 1)));
            if (!ok) {
                if (lane == 0) atomicExch(err, 1);
                bad = true;
                break;
            }
            const int4 inf = info[b];
            if (inf.x > 0 && act) {
                // slice bounds in records; the target leaf's own records (the
                // nearest, largest terms) are summed and folded on their own
                const int np = inf.x;
                const int jlo = (np * sl) / S, jhi = (np * (sl + 1)) / S;
                const int slo = inf.y, shi = inf.z;
                const ulonglong2 *pr = reinterpret_cast<const ulonglong2 *>(&buf[b][0]);
                const bool ownp = max(jlo, slo) < min(jhi, shi);
                p2p_pairs_pk<false, TPT>(jlo, min(jhi, slo), pr, tx, ty, tz, pacc, pcnt);
                if (ownp) {
                    p2p_fold_pk<TPT>(pacc, hls + threadIdx.x);
                    p2p_pairs_pk<true, TPT>(max(jlo, slo), min(jhi, shi), pr, tx, ty, tz, pacc, pcnt);
                    p2p_fold_pk<TPT>(pacc, hls + threadIdx.x);
                    pcnt = 0;
                }
                p2p_pairs_pk<false, TPT>(max(jlo, shi), jhi, pr, tx, ty, tz, pacc, pcnt);
                if (pcnt >= FMM_P2P_FOLD) {
                    p2p_fold_pk<TPT>(pacc, hls + threadIdx.x);
                    pcnt = 0;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[b]);
            cc++;
            if (inf.x == 0) break;
        }
        // after a timeout, copies that may still be in flight land before the
        // buffers are reused or released (bounded waits)
        if (bad && warp == 0 && lane == 0)
            for (int c = cc; c < pnext; c++) mbar_wait(&full[c % PR_NB], (uint32_t)((c / PR_NB) & 1));
        __syncthreads();  // every warp is past the last chunk: the buffers take the slice sums
        if (act) {
            p2p_fold_pk<TPT>(pacc, hls + threadIdx.x);
#pragma unroll
            for (int c = 0; c < 4 * TPT; c++)
                red2[(sl * R + row) * 4 * TPT + c] =
                    make_float2(hls[c * P2P_T + threadIdx.x], hls[(4 * TPT + c) * P2P_T + threadIdx.x]);
        }
        __syncthreads();
        if ((int)threadIdx.x < R) {
            // slices in fixed order, compensated in FP32 (TwoSum of the leading
            // parts, the trailing parts added), one conversion each
            float oh[4 * TPT], ol[4 * TPT];
#pragma unroll
            for (int c = 0; c < 4 * TPT; c++) oh[c] = ol[c] = 0.f;
            for (int s2 = 0; s2 < S; s2++)
#pragma unroll
                for (int c = 0; c < 4 * TPT; c++) {
                    const float2 v = red2[(s2 * R + threadIdx.x) * 4 * TPT + c];
                    acc2(oh[c], ol[c], v.x);
                    ol[c] += v.y;
                }
#pragma unroll
            for (int kk = 0; kk < TPT; kk++)
                if ((int)threadIdx.x + kk * R < nt)
                    near[t0 + threadIdx.x + kk * R] =
                        make_double4_32a((double)oh[4 * kk] + (double)ol[4 * kk], (double)oh[4 * kk + 1] + (double)ol[4 * kk + 1],
                                         (double)oh[4 * kk + 2] + (double)ol[4 * kk + 2],
                                         (double)oh[4 * kk + 3] + (double)ol[4 * kk + 3]);
        }
        // the slice sums (generic writes) are read, and ordered before the
        // bulk copies of the next pass or leaf that reuse the buffers
        fence_proxy_async();
        __syncthreads();
    }
}

template <int TPT>
__global__ void __launch_bounds__(P2P_T, FMM_P2P_MINB)
    p2p_pr_k(const float4 *__restrict__ xs, const float *__restrict__ pairs, const unsigned *__restrict__ pad,
             const unsigned *__restrict__ flag, const int *__restrict__ leaves, const int *__restrict__ begin,
             const int *__restrict__ end, const int *__restrict__ ptr, const int2 *__restrict__ runs_pr,
             const int *__restrict__ nrun, double4_32a *__restrict__ near, int *__restrict__ err)
{
    __shared__ PRShared<TPT> sh;
    p2p_pr_init(sh);
    int cc = 0;
    p2p_pr_leaf<TPT>(leaves[blockIdx.x], cc, sh, xs, pairs, pad, flag, begin, end, ptr, runs_pr, nrun, near, err);
}

// many systems: persistent blocks take (system, target leaf) items from the queue
template <int TPT>
__global__ void __launch_bounds__(P2P_T, FMM_P2P_MINB)
    batch_p2p_k(const BatchSys *__restrict__ sys, const int2 *__restrict__ items, int nitems, int *__restrict__ queue,
                int *__restrict__ err)
{
    __shared__ PRShared<TPT> sh;
    p2p_pr_init(sh);
    int cc = 0;
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(queue, 1);
        __syncthreads();
        const int it = sh.item;
        __syncthreads();  // every thread has the item before thread 0 takes the next
        if (it >= nitems) break;
        const int2 item = items[it];
        const BatchSys &S = sys[item.x];
        p2p_pr_leaf<TPT>(item.y, cc, sh, S.xs, S.pairs, S.pad, S.flag, S.begin, S.end, S.p2p_ptr, S.runs_pr, S.nrun,
                         S.near, err);
    }
}

void batch_p2p(int nsm, const BatchSys *sys, const int2 *items, int nitems, int *queue, int *err, cudaStream_t s)
{
    FMM_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(int), s));
    batch_p2p_k<FMM_P2P_TPT><<<nsm * FMM_P2P_MINB, P2P_T, 0, s>>>(sys, items, nitems, queue, err);
    check_launch("batch p2p");
}

// local expansions to zero; dependency counters to zero, except the root
// level of the downward pass, whose only cell is final after M2L
__global__ void batch_zero_k(int PP, const BatchSys *__restrict__ sys)
{
    const BatchSys &S = sys[blockIdx.y];
    const int64_t cnt = (int64_t)S.ncells * PP;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        S.L[i] = 0.f;
    if (blockIdx.x == 0 && threadIdx.x <= FMM_MAXLEVEL) {
        S.cnt_up[threadIdx.x] = 0u;
        S.cnt_dn[threadIdx.x] = threadIdx.x == 0 ? 1u : 0u;
    }
}

void batch_zero(int p, const BatchSys *sys, int nsys, cudaStream_t s)
{
    batch_zero_k<<<dim3(16, (unsigned)nsys), 256, 0, s>>>(p * p, sys);
    check_launch("batch zero");
}

// far + near back to each system's caller order: block b belongs to the
// system whose block range [blk0[s], blk0[s + 1]) holds it
__global__ void batch_combine_k(const BatchSys *__restrict__ sys, int nsys, const int *__restrict__ blk0)
{
    __shared__ int s_sys;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nsys - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (blk0[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_sys = lo;
    }
    __syncthreads();
    const BatchSys &S = sys[s_sys];
    const int64_t j = (int64_t)(blockIdx.x - blk0[s_sys]) * blockDim.x + threadIdx.x;
    if (j >= S.n) return;
    const int64_t i = S.inv[j];
    const double4_32a a = S.far[i], b = S.near[i];
    S.phi[j] = (float)(a.x + b.x);
    S.grad[3 * j + 0] = (float)(a.y + b.y);
    S.grad[3 * j + 1] = (float)(a.z + b.z);
    S.grad[3 * j + 2] = (float)(a.w + b.w);
}

void batch_combine(const BatchSys *sys, int nsys, const int *blk0, int nblocks, cudaStream_t s)
{
    if (nblocks == 0) return;
    batch_combine_k<<<nblocks, 256, 0, s>>>(sys, nsys, blk0);
    check_launch("batch combine");
}

void p2p_pairs_fill(fmm_ctx *h, cudaStream_t s)
{
    if (!h->pr_ready) return;
    const int64_t n = h->n;
    pr_fill_k<<<nblk(n, 256), 256, 0, s>>>(n, h->xs32.as<float4>(), h->pr_pad.as<unsigned>(), h->pr_flag.as<unsigned>(),
                                           h->pr_pairs.as<float>());
    count_launch(h);
    check_launch("p2p pairs");
}

void p2p_prepare(fmm_ctx *h, cudaStream_t s)
{
    h->pr_ready = false;
    if (!(h->precision == FMM_MIXED && h->dtype == FMM_F32) || h->nleaves == 0) return;
    const int64_t n = h->n;
    h->pr_flag.ensure(sizeof(unsigned) * (size_t)n);
    h->pr_pad.ensure(sizeof(unsigned) * (size_t)n);
    // at most one padding record half per leaf
    h->pr_pairs.ensure(sizeof(float) * 8 * (size_t)((n + h->nleaves + 1) / 2 + 1));
    h->p2p_runs_pr.ensure(sizeof(int2) * (size_t)std::max<int64_t>(h->n_p2p, 1));
    pr_flag_k<<<nblk(n, 256), 256, 0, s>>>(n, h->pcell.as<int>(), h->c_begin.as<int>(), h->c_end.as<int>(),
                                           h->pr_flag.as<unsigned>());
    count_launch(h);
    scan_exclusive_u32(h, h->pr_flag.as<unsigned>(), h->pr_pad.as<unsigned>(), n, nullptr, s);
    pr_runs_k<<<nblk(h->nleaves, 128), 128, 0, s>>>(h->nleaves, h->leaves.as<int>(), h->p2p_ptr.as<int>(),
                                                   h->p2p_nrun.as<int>(), h->p2p_runs.as<int2>(), h->pr_pad.as<unsigned>(),
                                                   h->pr_flag.as<unsigned>(), h->p2p_runs_pr.as<int2>());
    count_launch(h);
    check_launch("p2p pair runs");
    h->pr_ready = true;
    p2p_pairs_fill(h, s);
}

void near_field(fmm_ctx *h, cudaStream_t s)
{
    h->near.ensure(sizeof(double4_32a) * (size_t)h->n);
    if (h->nleaves == 0) return;
    const int *lv = h->leaves.as<int>(), *cb = h->c_begin.as<int>(), *ce = h->c_end.as<int>();
    const int *pp = h->p2p_ptr.as<int>(), *nr = h->p2p_nrun.as<int>();
    const int2 *ru = h->p2p_runs.as<int2>();
    double4_32a *out = h->near.as<double4_32a>();
    if (h->precision == FMM_FP64)
        p2p_k<double, false, 2><<<h->nleaves, P2P_T, 0, s>>>(h->xs64.as<double4_32a>(), nullptr, lv, cb, ce, pp, ru, nr, out);
    else if (h->dtype == FMM_F64)
        p2p_k<float, true, FMM_P2P_TPT><<<h->nleaves, P2P_T, 0, s>>>(h->xs32.as<float4>(), h->xs32lo.as<float4>(), lv, cb, ce, pp, ru,
                                                           nr, out);
    else if (h->pr_ready) {
        int *err = reinterpret_cast<int *>(h->m2l_misc.as<unsigned>() + 24 * (FMM_MAXLEVEL + 1) + 5);
        FMM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
        p2p_pr_k<FMM_P2P_TPT><<<h->nleaves, P2P_T, 0, s>>>(h->xs32.as<float4>(), h->pr_pairs.as<float>(),
                                                          h->pr_pad.as<unsigned>(), h->pr_flag.as<unsigned>(), lv, cb, ce,
                                                          pp, h->p2p_runs_pr.as<int2>(), nr, out, err);
    } else
        p2p_k<float, false, FMM_P2P_TPT><<<h->nleaves, P2P_T, 0, s>>>(h->xs32.as<float4>(), nullptr, lv, cb, ce, pp, ru, nr, out);
    count_launch(h);
    check_launch("p2p");
}

// ---------------------------------------------------------------------------
// far + near, back to the caller's particle order and element type
// ---------------------------------------------------------------------------
template <class OT>
__global__ void combine_k(const double4_32a *__restrict__ far, const double4_32a *__restrict__ near, const int *__restrict__ inv,
                          int64_t n, OT *__restrict__ phi, OT *__restrict__ grad)
{
    // one thread per particle in the caller's order: its sorted position is
    // read, the two 32-byte records gathered, and the outputs written in order
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t i = inv[j];
    const double4_32a a = far[i], b = near[i];
    phi[j] = (OT)(a.x + b.x);
    if (grad) {
        grad[3 * j + 0] = (OT)(a.y + b.y);
        grad[3 * j + 1] = (OT)(a.z + b.z);
        grad[3 * j + 2] = (OT)(a.w + b.w);
    }
}

void combine_unsort(fmm_ctx *h, void *phi, void *grad)
{
    if (h->dtype == FMM_F64)
        combine_k<double><<<nblk(h->n, 256), 256, 0, h->stream>>>(h->far.as<double4_32a>(), h->near.as<double4_32a>(),
                                                                  h->inv.as<int>(), h->n, (double *)phi, (double *)grad);
    else
        combine_k<float><<<nblk(h->n, 256), 256, 0, h->stream>>>(h->far.as<double4_32a>(), h->near.as<double4_32a>(),
                                                                 h->inv.as<int>(), h->n, (float *)phi, (float *)grad);
    count_launch(h);
    check_launch("combine");
}

// ---------------------------------------------------------------------------
// FP64 direct sum over all sources for a set of targets; the sources are
// split into nsplit ranges so that a few thousand targets still fill the GPU,
// and the partial sums are added in range order.
// ---------------------------------------------------------------------------
constexpr int DS_T = 128, DS_TILE = 256;

__global__ void __launch_bounds__(DS_T) direct_k(const double *__restrict__ x, const double *__restrict__ q, int64_t n,
                                                 const int64_t *__restrict__ tidx, int64_t nt, int64_t chunk,
                                                 double *__restrict__ part)
{
    __shared__ double4_32a sh[DS_TILE];
    const int64_t t = (int64_t)blockIdx.x * DS_T + threadIdx.x;
    const int split = blockIdx.y;
    const bool act = t < nt;
    const int64_t i = act ? (tidx ? tidx[t] : t) : 0;
    const double xi = act ? x[3 * i] : 0.0, yi = act ? x[3 * i + 1] : 0.0, zi = act ? x[3 * i + 2] : 0.0;
    const int64_t j0 = (int64_t)split * chunk, j1 = min(n, j0 + chunk);
    double p = 0, gx = 0, gy = 0, gz = 0;
    for (int64_t b = j0; b < j1; b += DS_TILE) {
        __syncthreads();
        for (int k = threadIdx.x; k < DS_TILE; k += DS_T) {
            const int64_t j = b + k;
            sh[k] = j < j1 ? make_double4_32a(x[3 * j], x[3 * j + 1], x[3 * j + 2], q[j]) : make_double4_32a(0, 0, 0, 0);
        }
        __syncthreads();
        const int m = (int)min((int64_t)DS_TILE, j1 - b);
        for (int k = 0; k < m; k++) {
            if (b + k == i) continue;
            const double4_32a s = sh[k];
            const double dx = xi - s.x, dy = yi - s.y, dz = zi - s.z;
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            const double r = sqrt(r2);
            const double qr = s.w / r;
            const double qr3 = qr / r2;
            p += qr;
            gx -= qr3 * dx;
            gy -= qr3 * dy;
            gz -= qr3 * dz;
        }
    }
    if (act) {
        double *o = part + ((size_t)split * nt + t) * 4;
        o[0] = p;
        o[1] = gx;
        o[2] = gy;
        o[3] = gz;
    }
}

__global__ void direct_reduce_k(const double *__restrict__ part, int nsplit, int64_t nt, double *__restrict__ phi,
                                double *__restrict__ grad)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double o[4] = {0, 0, 0, 0};
    for (int s = 0; s < nsplit; s++)
        for (int c = 0; c < 4; c++) o[c] += part[((size_t)s * nt + t) * 4 + c];
    phi[t] = o[0];
    if (grad) {
        grad[3 * t] = o[1];
        grad[3 * t + 1] = o[2];
        grad[3 * t + 2] = o[3];
    }
}

void direct_sum(fmm_ctx *h, const double *x, const double *q, int64_t n, const int64_t *tidx, int64_t nt, double *phi,
                double *grad)
{
    cudaStream_t s = h->stream;
    const int64_t tb = (nt + DS_T - 1) / DS_T;
    int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((4LL * h->nsm + tb - 1) / tb, (n + 4095) / 4096));
    nsplit = std::min(nsplit, 65535);
    const int64_t chunk = (n + nsplit - 1) / nsplit;
    h->direct_part.ensure(sizeof(double) * 4 * (size_t)nsplit * (size_t)nt);
    dim3 grid((unsigned)tb, (unsigned)nsplit);
    direct_k<<<grid, DS_T, 0, s>>>(x, q, n, tidx, nt, chunk, h->direct_part.as<double>());
    count_launch(h);
    direct_reduce_k<<<nblk(nt, 256), 256, 0, s>>>(h->direct_part.as<double>(), nsplit, nt, phi, grad);
    count_launch(h);
    check_launch("direct");
}

}  // namespace fmm
