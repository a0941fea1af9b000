// ohm_kernels.cu -- sm_103a kernels of the implicit ohmic-dissipation step
// (T. Matsumoto 2011, Sec. 2).  One thread block works on one 8^3-cell block: it stages the
// block and a one-cell halo (faces and edges; corners are never read by the stencil) in
// shared memory, from the same-grid neighbour blocks or, where the grid has no neighbour,
// from the block's coarse-fine ghost slot.
//
// Face flux (Eqs. 4-6, 9-11), kept scaled as Phi = 2 h F:
//   Phi_a^b = (eta_lo + eta_hi) * (T/4 - N),  N = B_b(hi) - B_b(lo)                 (Eq. 9)
//   T = B_a(lo+e_b) + B_a(hi+e_b) - B_a(lo-e_b) - B_a(hi-e_b)                         (Eq. 10)
// and the flux divergence (Eq. 8) is sum_a (Phi_a(+) - Phi_a(-)) / (2 h^2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "ohm_internal.h"

namespace ohm {

__device__ __forceinline__ int tix(int i, int j, int k) { return (k * TS + j) * TS + i; }

// batched inner iterations: block b belongs to an instance that is not iterated
__device__ __forceinline__ bool skip_block(const GridDev &g, int b) {
    return g.imask && !g.imask[g.inst_nblk ? b / g.inst_nblk : 0];
}

// ------------------------------------------------------------------ float-float arithmetic
// GB300 issues float64 at 1/58 of the float32 rate, so the outer residual of the mixed path
// runs on pairs of float32 values instead (Dekker 1971).  Every operation uses the explicitly
// rounded intrinsics, which the compiler never fuses into FMAs, so the error-free
// transformations stay exact:
//   two_sum (Knuth): s = fl(a + b) and the exact error of that addition;
//   fast_two_sum (Dekker): the same when |a| >= |b| (or a = 0), in three operations;
//   products: fl(a.hi b.hi) and its exact error from an FMA, plus the cross terms.
// Sums fold the trailing parts in before one renormalisation.  Their error is at most about
// 2^-47 (|a| + |b|): bounded against the operands, not the result, which is the measure the
// residual needs (its cancellation error is measured against |X|).
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dfloat(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

// float64 -> float-float by bit manipulation (no float64 instruction): hi carries the sign,
// the exponent and the leading 24 significand bits (truncated), lo the remaining 29 bits
// rounded to 24, so hi + lo keeps about 48 of the 53 bits.  Magnitudes outside the normal
// float32 range give lo = 0 and a signed hi: NaN stays NaN, infinities and finite values of
// 2^128 and above become infinite, values below 2^-126 become zero.
__device__ __forceinline__ dfloat split_double(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned int uh = (unsigned int)(u >> 32), ul = (unsigned int)u;
    const int e = (int)((uh >> 20) & 0x7ffu);  // biased float64 exponent
    const int fe = e - (1023 - 127);           // the same exponent biased for float32
    const unsigned int sgn = uh & 0x80000000u;
    if ((unsigned)(fe - 1) >= 254u) {
        const unsigned int nan = e == 0x7ff && ((uh & 0xfffffu) | ul) ? 0x400000u : 0u;
        return dfloat(__uint_as_float(fe >= 255 ? sgn | 0x7f800000u | nan : sgn));
    }
    const float hi = __uint_as_float(sgn | ((unsigned)fe << 23) | ((uh & 0xfffffu) << 3) | (ul >> 29));
    // lo = r 2^(e - 1075) for the 29 low significand bits r; where 2^(e - 1075) is below the
    // normal float32 range it is applied in two exact steps, 2^(e - 1075 + 64) and 2^-64
    const int k = e < 1075 - 126 ? 64 : 0;
    const float s1 = __uint_as_float((unsigned)(e - 1075 + k + 127) << 23);
    const float s2 = __uint_as_float((unsigned)(127 - k) << 23);
    const float lo = __fmul_rn(__fmul_rn(__uint2float_rn(ul & 0x1fffffffu), s1), s2);
    return dfloat(hi, sgn ? -lo : lo);
}

// Conversions used outside the float-float hot loop (flux registers, refluxing)
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(dfloat v) { return (double)v.hi + (double)v.lo; }
template <typename T>
__device__ __forceinline__ T from_double(double v) { return (T)v; }
template <>
__device__ __forceinline__ dfloat from_double<dfloat>(double v) {
    const float h = __double2float_rn(v);
    return dfloat(h, __double2float_rn(v - (double)h));
}
// staged tile value from a field value (float64 fields split for float-float tiles)
template <typename T, typename TS>
__device__ __forceinline__ T tile_val(TS v) {
    static_assert(sizeof(T) == sizeof(TS), "tile and field types differ in size");
    return v;
}
template <>
__device__ __forceinline__ dfloat tile_val<dfloat, double>(double v) { return split_double(v); }
// x / 4 (exact for every type)
__device__ __forceinline__ float quarter(float v) { return 0.25f * v; }
__device__ __forceinline__ double quarter(double v) { return 0.25 * v; }
__device__ __forceinline__ dfloat quarter(dfloat v) { return dfloat(0.25f * v.hi, 0.25f * v.lo); }
// leading value (the float32 or float64 approximation used for outputs and norms)
__device__ __forceinline__ float lead(float v) { return v; }
__device__ __forceinline__ double lead(double v) { return v; }
__device__ __forceinline__ float lead(dfloat v) { return v.hi; }
template <typename X>
struct Ident {
    using type = X;
};

// Shared-memory geometry of a staged 10^3 tile (block + 1-cell halo).  Rows along x are RS
// elements apart; PX is the row stride of the x-face flux array; tile x index ti sits at row
// offset OFF + ti.  float32 rows of 12 with OFF = 1 put the 8 interior cells of a row on an
// 8-byte boundary (staged as four 64-bit words); the compact tile (36 KB for the residual
// kernel) lets 4 thread blocks of 512 threads share an SM, which measured faster at 256^3
// (0.390 ms against 0.426 ms per residual + restriction) than rows padded to 24 floats, which
// avoid the 2-way bank conflicts of this layout but fit only 3 blocks per SM.  float64 kernels
// are bound by the float64 pipe and keep the compact stride.
template <typename T>
struct G10;
template <>
struct G10<float> {
    static constexpr int RS = 12, PX = 9, OFF = 1;
};
template <>
struct G10<double> {
    static constexpr int RS = 10, PX = 9, OFF = 0;
};
template <>
struct G10<dfloat> {
    static constexpr int RS = 10, PX = 9, OFF = 0;
};
// z-face planes are PZ apart: 72 for float32 (= 8 mod 32 banks, like the x- and y-face arrays
// and the tile planes, so a warp of 4 planes x 8 cells reads 32 distinct banks), 64 for float64
template <typename T>
struct Geo {
    static constexpr int RS = G10<T>::RS, PS = TS * RS, CS = TS * PS, PX = G10<T>::PX, OFF = G10<T>::OFF;
    static constexpr int PZ = sizeof(T) == 4 ? 72 : 64;
    static constexpr int PHI_X = 64 * PX;  // x faces per component
    static constexpr int PHI = 2 * PHI_X + 2 * 576 + 2 * 9 * PZ;
    __device__ static __forceinline__ int at(int i, int j, int k) { return k * PS + j * RS + i + OFF; }
    __device__ static __forceinline__ int xf(int fi, int j, int k) { return (k * 8 + j) * PX + fi; }
    __device__ static __forceinline__ int zf(int i, int j, int fk) { return fk * PZ + j * 8 + i; }
};

// 8 consecutive values of a block row (16-byte aligned in global memory) as vector loads
template <typename T>
struct Row8 {
    T v[8];
};
__device__ __forceinline__ Row8<float> load_row8(const float *__restrict__ p) {
    Row8<float> r;
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = a.z; r.v[3] = a.w;
    r.v[4] = b.x; r.v[5] = b.y; r.v[6] = b.z; r.v[7] = b.w;
    return r;
}
__device__ __forceinline__ Row8<double> load_row8(const double *__restrict__ p) {
    Row8<double> r;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p) + q);
        r.v[2 * q] = a.x;
        r.v[2 * q + 1] = a.y;
    }
    return r;
}

// Row-wise staging of a block and a halo of width HW (tile edge S = 8 + 2 HW; rows along x
// RS elements apart, planes S*RS, components S*S*RS), NC components of field F, from the 27
// neighbour ids in shared memory (snb, -1 = absent).  One task per (component, tile row):
// the 8 interior values of the row come from one block as vector loads, the HW halo cells at
// each end from the x-neighbours of that block.  Rows or cells of an absent neighbour come
// from `ghost` ([NC][10^3] compact, HW = 1 only) or are zero.  Values at the corners of the
// box are never read by the stencil and may be left stale.
template <typename T, typename TS>
__device__ __forceinline__ void store_row8(T *dst, const Row8<TS> &row, bool aligned16, bool aligned8 = false) {
    if constexpr (sizeof(T) == 4) {
        if (aligned16) {
            float4 *d4 = reinterpret_cast<float4 *>(dst);
            d4[0] = make_float4((float)row.v[0], (float)row.v[1], (float)row.v[2], (float)row.v[3]);
            d4[1] = make_float4((float)row.v[4], (float)row.v[5], (float)row.v[6], (float)row.v[7]);
            return;
        }
        if (aligned8) {
            float2 *d2 = reinterpret_cast<float2 *>(dst);
#pragma unroll
            for (int q = 0; q < 4; q++) d2[q] = make_float2((float)row.v[2 * q], (float)row.v[2 * q + 1]);
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < 8; q++) dst[q] = tile_val<T, TS>(row.v[q]);
}

// TS is the field's element type (T, or float64 for float-float tiles)
template <typename T, int NC, int HW, int RS, int OFF = 0, typename TS = T>
__device__ __forceinline__ void stage_rows(T *__restrict__ tile, const TS *__restrict__ F, const int *__restrict__ snb,
                                           const typename Ident<TS>::type *__restrict__ ghost) {
    constexpr int S = 8 + 2 * HW, S2 = S * S;
    constexpr bool A16 = sizeof(T) == 4 && (OFF + HW) % 4 == 0 && RS % 4 == 0;
    constexpr bool A8 = sizeof(T) == 4 && (OFF + HW) % 2 == 0 && RS % 2 == 0;
    for (int task = threadIdx.x; task < NC * S2; task += blockDim.x) {
        const int c = task / S2, rr = task - c * S2;
        const int tj = rr % S, tk = rr / S;
        const int lj = tj - HW, lk = tk - HW;
        const int dj = lj < 0 ? -1 : (lj > 7 ? 1 : 0), dk = lk < 0 ? -1 : (lk > 7 ? 1 : 0);
        const int sj = lj - 8 * dj, sk = lk - 8 * dk;
        T *dst = tile + c * (S2 * RS) + rr * RS + OFF;
        const TS *gh = ghost ? ghost + c * T3 + rr * S : nullptr;
        const int dcent = (dk + 1) * 9 + (dj + 1) * 3;
        const int src = snb[dcent + 1];
        if (src >= 0) {
            const Row8<TS> row = load_row8(F + ((size_t)src * NC + c) * B3 + (sk * 8 + sj) * 8);
            store_row8(dst + HW, row, A16, A8);
        } else {
#pragma unroll
            for (int q = 0; q < 8; q++) dst[HW + q] = gh ? tile_val<T, TS>(gh[HW + q]) : T(0);
        }
        const int slo = snb[dcent], shi = snb[dcent + 2];
        if constexpr (sizeof(T) == 4 && HW == 2 && OFF % 2 == 0 && RS % 2 == 0) {
          if (slo >= 0 && shi >= 0) {
            // two-cell halos as 8-byte words (cells 6,7 of the x- neighbour, 0,1 of the x+ one)
            const float2 lo = __ldg(reinterpret_cast<const float2 *>(F + ((size_t)slo * NC + c) * B3 + (sk * 8 + sj) * 8 + 6));
            const float2 hi = __ldg(reinterpret_cast<const float2 *>(F + ((size_t)shi * NC + c) * B3 + (sk * 8 + sj) * 8));
            *reinterpret_cast<float2 *>(dst) = lo;
            *reinterpret_cast<float2 *>(dst + HW + 8) = hi;
            continue;
          }
        }
#pragma unroll
        for (int h = 0; h < HW; h++) {
            // low end: cells 8-HW+h of the x- neighbour; high end: cells h of the x+ neighbour
            dst[h] = slo >= 0 ? tile_val<T, TS>(F[((size_t)slo * NC + c) * B3 + (sk * 8 + sj) * 8 + 8 - HW + h])
                              : (gh ? tile_val<T, TS>(gh[h]) : T(0));
            dst[HW + 8 + h] = shi >= 0 ? tile_val<T, TS>(F[((size_t)shi * NC + c) * B3 + (sk * 8 + sj) * 8 + h])
                                       : (gh ? tile_val<T, TS>(gh[HW + 8 + h]) : T(0));
        }
    }
}

// Element-wise staging, same tile layout as stage_rows: consecutive threads take consecutive
// cells of a tile row, so global loads are coalesced along x and shared-memory stores of a
// warp fall on consecutive addresses (stage_rows, one thread per row, stores 32 different
// rows at the same column at once, which for padded row strides hits few banks).
template <typename T, int NC, int HW, int RS>
__device__ __forceinline__ void stage_cells(T *__restrict__ tile, const T *__restrict__ F, const int *__restrict__ snb,
                                            const T *__restrict__ ghost) {
    constexpr int S = 8 + 2 * HW, S2 = S * S, S3 = S2 * S;
    for (int e = threadIdx.x; e < S3; e += blockDim.x) {
        const int tk = e / S2, rem = e - tk * S2, tj = rem / S, ti = rem - tj * S;
        const int li = ti - HW, lj = tj - HW, lk = tk - HW;
        const int di = li < 0 ? -1 : (li > 7 ? 1 : 0), dj = lj < 0 ? -1 : (lj > 7 ? 1 : 0), dk = lk < 0 ? -1 : (lk > 7 ? 1 : 0);
        const int src = snb[(dk + 1) * 9 + (dj + 1) * 3 + (di + 1)];
        const int dst = (tk * S + tj) * RS + ti;
        if (src >= 0) {
            const T *p = F + (size_t)src * NC * B3 + ((lk - 8 * dk) * 8 + (lj - 8 * dj)) * 8 + (li - 8 * di);
#pragma unroll
            for (int c = 0; c < NC; c++) tile[c * S2 * RS + dst] = p[c * B3];
        } else {
#pragma unroll
            for (int c = 0; c < NC; c++) tile[c * S2 * RS + dst] = ghost ? ghost[c * T3 + e] : T(0);
        }
    }
}

// neighbour ids of block b into shared memory (call before stage_rows, then __syncthreads)
__device__ __forceinline__ void stage_nbr(int *snb, const int *__restrict__ nbr, int b) {
    if (threadIdx.x < 27) snb[threadIdx.x] = __ldg(nbr + b * 27 + threadIdx.x);
}

// Phi = 2hF for the face between tile cells p (low) and p + sa, axis a (Eqs. 4-6, 9-11).
// The two flux components are the axes other than a in ascending order, with tile strides
// s1 and s2; components of the tile are cs elements apart.
template <typename T>
__device__ __forceinline__ void face_phi_s(const T *__restrict__ tB, const T *__restrict__ tE, int p, int a, int sa,
                                           int s1, int s2, int cs, T &phi1, T &phi2) {
    const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;
    const T es = tE[p] + tE[p + sa];
    const T *Ba = tB + a * cs;
    const T *B1 = tB + b1 * cs;
    const T *B2 = tB + b2 * cs;
    T n1 = B1[p + sa] - B1[p];
    T t1 = (Ba[p + sa + s1] + Ba[p + s1]) - (Ba[p + sa - s1] + Ba[p - s1]);
    phi1 = es * (quarter(t1) - n1);
    T n2 = B2[p + sa] - B2[p];
    T t2 = (Ba[p + sa + s2] + Ba[p + s2]) - (Ba[p + sa - s2] + Ba[p - s2]);
    phi2 = es * (quarter(t2) - n2);
}

// Faces of a 10^3 tile along axis a from the low tile cell p, in the geometry of T
template <typename T>
__device__ __forceinline__ void face10(const T *__restrict__ tB, const T *__restrict__ tE, int p, int a, T &p1, T &p2) {
    using G = Geo<T>;
    if (a == 0)
        face_phi_s(tB, tE, p, 0, 1, G::RS, G::PS, G::CS, p1, p2);
    else if (a == 1)
        face_phi_s(tB, tE, p, 1, G::RS, 1, G::PS, G::CS, p1, p2);
    else
        face_phi_s(tB, tE, p, 2, G::PS, 1, G::RS, G::CS, p1, p2);
}

// Offsets of the six flux arrays: x faces [2 comps][64 rows][PX] (index xf), y faces
// [2][8][9][8] ((k*9+fj)*8+i), z faces [2][9][PZ] (index zf).
template <typename T>
__device__ __forceinline__ int phi_base(int ax, int comp) {
    using G = Geo<T>;
    return ax == 0 ? comp * G::PHI_X : (ax == 1 ? 2 * G::PHI_X + comp * 576 : 2 * G::PHI_X + 2 * 576 + comp * 9 * G::PZ);
}

// Cell of thread t in the 512-thread stencil kernels.  float32: a warp takes one row index j of
// 4 consecutive planes (i fastest), whose tile and face-array offsets fall on 32 distinct banks
// for the compact strides above; float64 keeps i + 8 j + 64 k.
template <typename T>
__device__ __forceinline__ void cell_of_thread(int t, int &i, int &j, int &k) {
    if (sizeof(T) == 4) {
        i = t & 7;
        k = ((t >> 3) & 3) + 4 * (t >> 8);
        j = (t >> 5) & 7;
    } else {
        i = t & 7;
        j = (t >> 3) & 7;
        k = t >> 6;
    }
}

// All 1728 face fluxes of a staged block (512 threads): thread (i,j,k) computes the low x, y
// and z faces of its cell, then threads 0..191 compute the 3 x 64 faces of the high planes.
template <typename T>
__device__ __forceinline__ void all_faces_512(const T *__restrict__ tB, const T *__restrict__ tE, T *__restrict__ phi) {
    using G = Geo<T>;
    const int t = threadIdx.x;
    int i, j, k;
    cell_of_thread<T>(t, i, j, k);
    const int p = G::at(i + 1, j + 1, k + 1);
    T p1, p2;
    face10(tB, tE, p - 1, 0, p1, p2);
    phi[G::xf(i, j, k)] = p1;
    phi[G::PHI_X + G::xf(i, j, k)] = p2;
    face10(tB, tE, p - G::RS, 1, p1, p2);
    phi[phi_base<T>(1, 0) + (k * 9 + j) * 8 + i] = p1;
    phi[phi_base<T>(1, 1) + (k * 9 + j) * 8 + i] = p2;
    face10(tB, tE, p - G::PS, 2, p1, p2);
    phi[phi_base<T>(2, 0) + G::zf(i, j, k)] = p1;
    phi[phi_base<T>(2, 1) + G::zf(i, j, k)] = p2;
    if (t < 192) {
        const int ax = t >> 6, u = t & 7, v = (t >> 3) & 7;
        if (ax == 0) {  // x = 8 plane: (j, k) = (u, v)
            face10(tB, tE, G::at(8, u + 1, v + 1), 0, p1, p2);
            phi[G::xf(8, u, v)] = p1;
            phi[G::PHI_X + G::xf(8, u, v)] = p2;
        } else if (ax == 1) {  // y = 8 plane: (i, k) = (u, v)
            face10(tB, tE, G::at(u + 1, 8, v + 1), 1, p1, p2);
            phi[phi_base<T>(1, 0) + (v * 9 + 8) * 8 + u] = p1;
            phi[phi_base<T>(1, 1) + (v * 9 + 8) * 8 + u] = p2;
        } else {  // z = 8 plane: (i, j) = (u, v)
            face10(tB, tE, G::at(u + 1, v + 1, 8), 2, p1, p2);
            phi[phi_base<T>(2, 0) + G::zf(u, v, 8)] = p1;
            phi[phi_base<T>(2, 1) + G::zf(u, v, 8)] = p2;
        }
    }
}

// float64 face fluxes with shared pair sums.  The tangential term of Eq. 10 is a difference of
// two pair sums across the face, P_a(q) = B_a(q) + B_a(q + e_a), taken one cell apart along the
// flux component's axis; every pair sum serves two faces, so computing the 2592 sums of a block
// once (one float64 addition each) saves two additions per face flux, a fifth of the float64
// work of the composite operator.  The sums are the same additions in the same order as in
// face_phi_s, so the fluxes are bit-identical.  P holds, per axis a, [9 faces][10][10] sums over
// the face's tile coordinates (u, v) along the two other axes in ascending order (corners unused).
constexpr int PSUM = 3 * 900;
__device__ __forceinline__ void pair_sums_512(const double *__restrict__ tB, double *__restrict__ P) {
    using G = Geo<double>;
    for (int e = threadIdx.x; e < PSUM; e += blockDim.x) {
        const int a = e / 900, r = e - a * 900, fn = r / 100, v = (r / 10) % 10, u = r % 10;
        if ((u == 0 || u == 9) && (v == 0 || v == 9)) continue;  // corners: never staged, never read
        int p, sa;
        if (a == 0) { p = G::at(fn, u, v) ; sa = 1; }           // x faces: (u, v) = (y, z)
        else if (a == 1) { p = G::at(u, fn, v); sa = G::RS; }  // y faces: (u, v) = (x, z)
        else { p = G::at(u, v, fn); sa = G::PS; }              // z faces: (u, v) = (x, y)
        const double *Ba = tB + a * G::CS;
        P[e] = Ba[p + sa] + Ba[p];
    }
}

// Phi of the face with low tile cell p along axis a (tile tangential coordinates u0, v0), from
// the pair sums; the normal differences and eta as in face_phi_s.
__device__ __forceinline__ void face_phi_p(const double *__restrict__ tB, const double *__restrict__ tE,
                                           const double *__restrict__ P, int p, int a, int fn, int u0, int v0,
                                           double &phi1, double &phi2) {
    using G = Geo<double>;
    const int sa = a == 0 ? 1 : (a == 1 ? G::RS : G::PS);
    const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;
    const double es = tE[p] + tE[p + sa];
    const double *Pa = P + a * 900 + fn * 100;
    const double *B1 = tB + b1 * G::CS;
    const double *B2 = tB + b2 * G::CS;
    const double n1 = B1[p + sa] - B1[p];
    const double t1 = Pa[v0 * 10 + u0 + 1] - Pa[v0 * 10 + u0 - 1];
    phi1 = es * (quarter(t1) - n1);
    const double n2 = B2[p + sa] - B2[p];
    const double t2 = Pa[(v0 + 1) * 10 + u0] - Pa[(v0 - 1) * 10 + u0];
    phi2 = es * (quarter(t2) - n2);
}

// all_faces_512 for float64 with the pair sums (call after pair_sums_512 and a barrier)
__device__ __forceinline__ void all_faces_512_p(const double *__restrict__ tB, const double *__restrict__ tE,
                                                const double *__restrict__ P, double *__restrict__ phi) {
    using G = Geo<double>;
    const int t = threadIdx.x;
    int i, j, k;
    cell_of_thread<double>(t, i, j, k);
    const int p = G::at(i + 1, j + 1, k + 1);
    double p1, p2;
    face_phi_p(tB, tE, P, p - 1, 0, i, j + 1, k + 1, p1, p2);
    phi[G::xf(i, j, k)] = p1;
    phi[G::PHI_X + G::xf(i, j, k)] = p2;
    face_phi_p(tB, tE, P, p - G::RS, 1, j, i + 1, k + 1, p1, p2);
    phi[phi_base<double>(1, 0) + (k * 9 + j) * 8 + i] = p1;
    phi[phi_base<double>(1, 1) + (k * 9 + j) * 8 + i] = p2;
    face_phi_p(tB, tE, P, p - G::PS, 2, k, i + 1, j + 1, p1, p2);
    phi[phi_base<double>(2, 0) + G::zf(i, j, k)] = p1;
    phi[phi_base<double>(2, 1) + G::zf(i, j, k)] = p2;
    if (t < 192) {
        const int ax = t >> 6, u = t & 7, v = (t >> 3) & 7;
        if (ax == 0) {  // x = 8 plane: (j, k) = (u, v)
            face_phi_p(tB, tE, P, G::at(8, u + 1, v + 1), 0, 8, u + 1, v + 1, p1, p2);
            phi[G::xf(8, u, v)] = p1;
            phi[G::PHI_X + G::xf(8, u, v)] = p2;
        } else if (ax == 1) {  // y = 8 plane: (i, k) = (u, v)
            face_phi_p(tB, tE, P, G::at(u + 1, 8, v + 1), 1, 8, u + 1, v + 1, p1, p2);
            phi[phi_base<double>(1, 0) + (v * 9 + 8) * 8 + u] = p1;
            phi[phi_base<double>(1, 1) + (v * 9 + 8) * 8 + u] = p2;
        } else {  // z = 8 plane: (i, j) = (u, v)
            face_phi_p(tB, tE, P, G::at(u + 1, v + 1, 8), 2, 8, u + 1, v + 1, p1, p2);
            phi[phi_base<double>(2, 0) + G::zf(u, v, 8)] = p1;
            phi[phi_base<double>(2, 1) + G::zf(u, v, 8)] = p2;
        }
    }
}

// sum_a (Phi_a(+) - Phi_a(-)) at cell (i,j,k) for the three components
template <typename T>
__device__ __forceinline__ void cell_div(const T *__restrict__ phi, int i, int j, int k, T &dx, T &dy, T &dz) {
    using G = Geo<T>;
    const T *px0 = phi, *px1 = phi + G::PHI_X;                                // x faces: comps y, z
    const T *py0 = phi + phi_base<T>(1, 0), *py1 = phi + phi_base<T>(1, 1);  // y faces: comps x, z
    const T *pz0 = phi + phi_base<T>(2, 0), *pz1 = phi + phi_base<T>(2, 1);  // z faces: comps x, y
    const int xl = G::xf(i, j, k), yl = (k * 9 + j) * 8 + i, zl = G::zf(i, j, k);
    dx = (py0[yl + 8] - py0[yl]) + (pz0[zl + G::PZ] - pz0[zl]);
    dy = (px0[xl + 1] - px0[xl]) + (pz1[zl + G::PZ] - pz1[zl]);
    dz = (px1[xl + 1] - px1[xl]) + (py1[yl + 8] - py1[yl]);
}

// index in the flux arrays of the boundary-plane face (u, v) of side s = 2a + hi, where
// (u, v) run over the two axes other than a in ascending order
template <typename T>
__device__ __forceinline__ int plane_face(int a, int hi, int comp, int u, int v) {
    using G = Geo<T>;
    if (a == 0) return phi_base<T>(0, comp) + G::xf(hi ? 8 : 0, u, v);
    if (a == 1) return phi_base<T>(1, comp) + (v * 9 + (hi ? 8 : 0)) * 8 + u;
    return phi_base<T>(2, comp) + G::zf(u, v, hi ? 8 : 0);
}

// Block-wide sum / max in a fixed order (deterministic); the result is valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    if (w == 0) {
        s = threadIdx.x < nw ? red[threadIdx.x] : T(0);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

template <typename T>
__device__ __forceinline__ T block_max(T v, T *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    if (w == 0) {
        s = threadIdx.x < nw ? red[threadIdx.x] : T(0);
        for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    }
    return s;
}

// ------------------------------------------------------------------ composite operator
// Computed in TC: float64 for the outer residual and the source of the float64 path, float-float
// (dfloat, from float64 fields) for those of the mixed path, float32 for the inner residual of
// mixed precision; refluxed fluxes travel through float64 registers.
template <typename TC>
struct CompTypes {
    using In = TC;   // element type of X, eta and the ghosts
    using Acc = TC;  // norm accumulation
    static constexpr int minb = sizeof(TC) == 4 ? 4 : 1;
};
template <>
struct CompTypes<dfloat> {
    using In = double;
    using Acc = float;
    static constexpr int minb = 3;
};

template <typename TC, typename TO, bool NORMS, typename YT = TC>
__global__ void __launch_bounds__(512, CompTypes<TC>::minb)
    k_composite(GridDev g, const typename CompTypes<TC>::In *__restrict__ X, const YT *__restrict__ Y,
                const typename CompTypes<TC>::In *__restrict__ eta, const typename CompTypes<TC>::In *__restrict__ Gx,
                const typename CompTypes<TC>::In *__restrict__ Geta, TC a, TC coef, TC d, TO *__restrict__ out,
                TO *__restrict__ out2, double *__restrict__ reg, const int *__restrict__ rsrc_tab,
                double *__restrict__ partials, double vol, TC *__restrict__ outS, TC coef2, double inv2h, double twoh, bool ymx) {
    using G = Geo<TC>;
    using TA = typename CompTypes<TC>::Acc;
    using TM = typename std::conditional<sizeof(TO) == 4, float, TA>::type;  // max |out| from the output copy
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC *tB = reinterpret_cast<TC *>(smem_raw);
    TC *tE = tB + 3 * G::CS;
    TC *phi = tE + G::CS;
    __shared__ int snb[27];
    const int b = blockIdx.x;
    if (skip_block(g, b)) return;
    if (g.covered && g.covered[b]) {
        if (NORMS && threadIdx.x < 3) partials[b * 3 + threadIdx.x] = 0.0;
        return;
    }
    const int slot = g.gslot ? g.gslot[b] : -1;
    stage_nbr(snb, g.nbr, b);
    __syncthreads();
    stage_rows<TC, 3, 1, G::RS, G::OFF>(tB, X, snb, slot >= 0 && Gx ? Gx + (size_t)slot * 3 * T3 : nullptr);
    stage_rows<TC, 1, 1, G::RS, G::OFF>(tE, eta, snb, slot >= 0 && Geta ? Geta + (size_t)slot * T3 : nullptr);
    __syncthreads();
    if constexpr (std::is_same<TC, double>::value) {
        double *P = phi + G::PHI;  // pair sums after the flux arrays
        pair_sums_512(tB, P);
        __syncthreads();
        all_faces_512_p(tB, tE, P, phi);
    } else {
        all_faces_512(tB, tE, phi);
    }
    __syncthreads();
    // flux registers: faces with no same-level neighbour publish F = Phi / (2h) (inv2h = 1 / (2h)
    // and twoh = 2h come from the host: a float64 division here would cost the float32 kernels
    // dearly on a GPU with few float64 units)
    if (g.freg) {
        for (int s = 0; s < 6; s++) {
            int slotr = g.freg[b * 6 + s];
            if (slotr < 0) continue;
            int ax = s >> 1, hi = s & 1;
            for (int q = threadIdx.x; q < 128; q += blockDim.x) {
                int comp = q >> 6, uv = q & 63;
                reg[(size_t)slotr * 128 + q] = to_double(phi[plane_face<TC>(ax, hi, comp, uv & 7, uv >> 3)]) * inv2h;
            }
        }
    }
    // refluxing: faces next to a covered block take 2h * (mean of the four fine fluxes)
    if (g.rsrc) {
        for (int s = 0; s < 6; s++) {
            int src = g.rsrc[b * 6 + s];
            if (src < 0) continue;
            int ax = s >> 1, hi = s & 1;
            for (int q = threadIdx.x; q < 128; q += blockDim.x) {
                int comp = q >> 6, u = q & 7, v = (q >> 3) & 7;
                int fslot = rsrc_tab[src * 4 + (v >> 2) * 2 + (u >> 2)];
                const double *R = reg + (size_t)fslot * 128 + comp * 64;
                int fu = 2 * (u & 3), fv = 2 * (v & 3);
                double m = 0.25 * ((R[fv * 8 + fu] + R[fv * 8 + fu + 1]) + (R[(fv + 1) * 8 + fu] + R[(fv + 1) * 8 + fu + 1]));
                phi[plane_face<TC>(ax, hi, comp, u, v)] = from_double<TC>(m * twoh);
            }
        }
        __syncthreads();  // refluxed faces before the divergence (g.rsrc is uniform: legal)
    }
    int i, j, k;
    cell_of_thread<TC>(threadIdx.x, i, j, k);
    const int cell = (k * 8 + j) * 8 + i;
    TC dv[3];
    cell_div(phi, i, j, k, dv[0], dv[1], dv[2]);
    TA sr = 0, ss = 0;
    TM mx = 0;
    const int p = G::at(i + 1, j + 1, k + 1);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        size_t id = ((size_t)b * 3 + c) * B3 + cell;
        TC y = Y ? tile_val<TC, YT>(Y[id]) : TC(0);
        // ymx: a = -1, d = 1 (a residual), one operation less per component
        TC o = ymx ? (y - tB[c * G::CS + p]) + coef * dv[c] : a * tB[c * G::CS + p] + coef * dv[c] + d * y;
        if (sizeof(TC) == 8 && outS) {  // o is the source; the residual of X against it is coef2 divF(X)
            outS[id] = o;
            y = o;
            o = coef2 * dv[c];
        }
        const TA ol = lead(o);
        const TO oo = (TO)ol;
        out[id] = oo;
        if (out2) out2[id] = oo;
        if constexpr (NORMS) {
            const TA yl = lead(y);
            sr += ol * ol;
            ss += yl * yl;
            mx = fmax(mx, fabs((TM)oo));
        }
    }
    if constexpr (NORMS) {
        // Block sums through shared memory (the flux arrays are free now): warps 0, 1, 2 each
        // reduce one of the 512-entry columns (16 entries per lane, then 5 shuffle levels), so
        // the float64 pipe sees 21 additions per warp instead of 15 per thread.  Fixed order.
        __syncthreads();
        TA *rs = reinterpret_cast<TA *>(phi);
        TM *rm = reinterpret_cast<TM *>(rs + 2 * B3);
        rs[threadIdx.x] = sr;
        rs[B3 + threadIdx.x] = ss;
        rm[threadIdx.x] = mx;
        __syncthreads();
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (w < 2) {
            const TA *src = rs + w * B3;
            TA v = src[lane];
#pragma unroll
            for (int q = 1; q < B3 / 32; q++) v += src[lane + 32 * q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) partials[b * 3 + w] = (double)v * vol;
        } else if (w == 2) {
            TM v = rm[lane];
#pragma unroll
            for (int q = 1; q < B3 / 32; q++) v = fmax(v, rm[lane + 32 * q]);
            for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) partials[b * 3 + 2] = (double)v;
        }
    }
}

template <typename TC, typename TO, typename YT = TC>
static cudaError_t launch_composite_t(const GridDev &g, const typename CompTypes<TC>::In *X, const YT *Y,
                                     const typename CompTypes<TC>::In *eta, const typename CompTypes<TC>::In *Gx,
                                     const typename CompTypes<TC>::In *Geta, TC a, TC coef, TC d, TO *out, TO *out2,
                                     double *reg, const int *rsrc_tab, double *partials, double vol, cudaStream_t s,
                                     TC *outS, TC coef2, bool ymx) {
    if (g.nblk == 0) return cudaSuccess;
    const size_t sm = (4 * Geo<TC>::CS + Geo<TC>::PHI + (std::is_same<TC, double>::value ? PSUM : 0)) * sizeof(TC);
    // set once per process (thread-safe static initialisation)
    static const bool attr = (cudaFuncSetAttribute(k_composite<TC, TO, true, YT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                              cudaFuncSetAttribute(k_composite<TC, TO, false, YT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                              true);
    (void)attr;
    if (partials)  // with norm partials (the block reductions are compiled out otherwise)
        k_composite<TC, TO, true, YT><<<g.nblk, 512, sm, s>>>(g, X, Y, eta, Gx, Geta, a, coef, d, out, out2, reg, rsrc_tab,
                                                              partials, vol, outS, coef2, 0.5 / g.h, 2.0 * g.h, ymx);
    else
        k_composite<TC, TO, false, YT><<<g.nblk, 512, sm, s>>>(g, X, Y, eta, Gx, Geta, a, coef, d, out, out2, reg,
                                                               rsrc_tab, partials, vol, outS, coef2, 0.5 / g.h, 2.0 * g.h,
                                                               ymx);
    return cudaGetLastError();
}

template <typename TC, typename TO>
cudaError_t launch_composite(const GridDev &g, const TC *X, const TC *Y, const TC *eta, const TC *Gx, const TC *Geta,
                             double a, double c, double d, TO *out, TO *out2, double *reg, const int *rsrc_tab,
                             double *partials, double vol, cudaStream_t s, double *outS, double c2) {
    const double coef = c / (2.0 * g.h * g.h), coef2 = c2 / (2.0 * g.h * g.h);
    // outS is set only for TC = float64 (the source of a step)
    return launch_composite_t<TC, TO>(g, X, Y, eta, Gx, Geta, (TC)a, (TC)coef, (TC)d, out, out2, reg, rsrc_tab,
                                      partials, vol, s, reinterpret_cast<TC *>(outS), (TC)coef2, a == -1.0 && d == 1.0);
}

// float64 coefficient as float-float (hi = nearest float32, lo = nearest float32 to the rest)
static dfloat df_from_host(double v) {
    const float h = (float)v;
    return dfloat(h, (float)(v - (double)h));
}

cudaError_t launch_composite_df(const GridDev &g, const double *X, const dfloat *Y, const double *eta,
                                const double *Gx, const double *Geta, double a, double c, double d, float *out,
                                float *out2, double *reg, const int *rsrc_tab, double *partials, double vol,
                                cudaStream_t s, dfloat *outS, double c2) {
    const double coef = c / (2.0 * g.h * g.h), coef2 = c2 / (2.0 * g.h * g.h);
    return launch_composite_t<dfloat, float>(g, X, Y, eta, Gx, Geta, df_from_host(a), df_from_host(coef),
                                             df_from_host(d), out, out2, reg, rsrc_tab, partials, vol, s, outS,
                                             df_from_host(coef2), a == -1.0 && d == 1.0);
}
cudaError_t launch_composite_df(const GridDev &g, const double *X, const double *Y, const double *eta,
                                const double *Gx, const double *Geta, double a, double c, double d, float *out,
                                float *out2, double *reg, const int *rsrc_tab, double *partials, double vol,
                                cudaStream_t s) {
    const double coef = c / (2.0 * g.h * g.h);
    return launch_composite_t<dfloat, float, double>(g, X, Y, eta, Gx, Geta, df_from_host(a), df_from_host(coef),
                                                     df_from_host(d), out, out2, reg, rsrc_tab, partials, vol, s,
                                                     nullptr, dfloat(), a == -1.0 && d == 1.0);
}
#define INST_COMPOSITE(TC, TO)                                                                                        \
    template cudaError_t launch_composite<TC, TO>(const GridDev &, const TC *, const TC *, const TC *, const TC *,     \
                                                  const TC *, double, double, double, TO *, TO *, double *, const int *, \
                                                  double *, double, cudaStream_t, double *, double);
INST_COMPOSITE(double, double)
INST_COMPOSITE(double, float)
INST_COMPOSITE(float, float)

// ------------------------------------------------------------------ red-black smoothing
// One colour pass (Eq. 19): colour cells get e + (r - e - lamdt divF(e)) * inv, the other
// colour is copied; e_in and e_out are distinct buffers so every update reads the pre-pass
// state (Jacobi within a colour).  256 threads, one per colour cell.
template <typename T>
__global__ void __launch_bounds__(256) k_smooth(GridDev g, const T *__restrict__ e_in, T *__restrict__ e_out,
                                                const T *__restrict__ r, const T *__restrict__ eta,
                                                const T *__restrict__ inv, const T *__restrict__ Ge,
                                                const T *__restrict__ Geta, T coef, int colour) {
    using G = Geo<T>;
    __shared__ __align__(16) T tB[3 * G::CS];
    __shared__ __align__(16) T tE[G::CS];
    __shared__ int snb[27];
    const int b = blockIdx.x;
    if (skip_block(g, b)) return;
    const int slot = g.gslot ? g.gslot[b] : -1;
    stage_nbr(snb, g.nbr, b);
    __syncthreads();
    stage_rows<T, 3, 1, G::RS, G::OFF>(tB, e_in, snb, slot >= 0 && Ge ? Ge + (size_t)slot * 3 * T3 : nullptr);
    stage_rows<T, 1, 1, G::RS, G::OFF>(tE, eta, snb, slot >= 0 && Geta ? Geta + (size_t)slot * T3 : nullptr);
    __syncthreads();
    const int t = threadIdx.x;
    const int k = t >> 5, j = (t >> 2) & 7;
    const int ic = 2 * (t & 3) + ((j + k + colour) & 1);      // colour cell
    const int io = 2 * (t & 3) + ((j + k + colour + 1) & 1);  // other colour
    const int p = G::at(ic + 1, j + 1, k + 1);
    T xl1, xl2, xh1, xh2, yl1, yl2, yh1, yh2, zl1, zl2, zh1, zh2;
    face10(tB, tE, p - 1, 0, xl1, xl2);
    face10(tB, tE, p, 0, xh1, xh2);
    face10(tB, tE, p - G::RS, 1, yl1, yl2);
    face10(tB, tE, p, 1, yh1, yh2);
    face10(tB, tE, p - G::PS, 2, zl1, zl2);
    face10(tB, tE, p, 2, zh1, zh2);
    T dv[3];
    dv[0] = (yh1 - yl1) + (zh1 - zl1);
    dv[1] = (xh1 - xl1) + (zh2 - zl2);
    dv[2] = (xh2 - xl2) + (yh2 - yl2);
    const int cc = (k * 8 + j) * 8 + ic, co = (k * 8 + j) * 8 + io;
    const int po = G::at(io + 1, j + 1, k + 1);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        size_t base = ((size_t)b * 3 + c) * B3;
        T ev = tB[c * G::CS + p];
        T res = r[base + cc] - ev - coef * dv[c];
        e_out[base + cc] = ev + res * inv[base + cc];
        e_out[base + co] = tB[c * G::CS + po];
    }
}

template <typename T>
cudaError_t launch_smooth(const GridDev &g, const T *e_in, T *e_out, const T *r, const T *eta, const T *inv,
                          const T *Ge, const T *Geta, double lamdt, int colour, cudaStream_t s) {
    if (g.nblk == 0) return cudaSuccess;
    T coef = (T)(lamdt / (2.0 * g.h * g.h));
    k_smooth<T><<<g.nblk, 256, 0, s>>>(g, e_in, e_out, r, eta, inv, Ge, Geta, coef, colour);
    return cudaGetLastError();
}
template cudaError_t launch_smooth<double>(const GridDev &, const double *, double *, const double *, const double *,
                                           const double *, const double *, const double *, double, int, cudaStream_t);
template cudaError_t launch_smooth<float>(const GridDev &, const float *, float *, const float *, const float *,
                                          const float *, const float *, const float *, double, int, cudaStream_t);

// ------------------------------------------------------------------ fused red + black sweep
// One full red-black sweep in one launch, for grids whose blocks have every neighbour (no
// coarse-fine ghosts).  The block and a 2-cell halo (12^3, all 26 neighbours) are staged;
// red cells of the block and of its 1-cell ring get their update from the pre-sweep state,
// then the block's black cells are updated from the post-red state.  The ring updates are
// the ones the neighbouring blocks compute, in the same order with the same arithmetic, so
// the result equals two global colour passes.  The inverse diagonal is formed on the fly
// from eta (Eqs. 21-23).  e_in and e_out are distinct buffers.
// The 12^3 tile is compact (rows 12 elements apart): 8 rows of 4 same-colour cells (stride 2,
// the warp pattern of the block's cells) still fall on 32 distinct float32 banks, and the
// tile (4 x 6.75 KB for float32) leaves room for 6 thread blocks per SM.  The sweep is bound by
// latency more than by shared-memory bandwidth: a padded tile (rows 20 apart, fewer bank
// conflicts on the ring) measured slower at 256^3 (0.46 ms against 0.43 ms per sweep) because
// it allows only 4 thread blocks per SM.
template <typename T>
struct G12 {
    static constexpr int S = 12, RRS = 12, PS = S * RRS, CS = S * PS, OFF = 0;
    __device__ static __forceinline__ int at(int i, int j, int k) { return k * PS + j * RRS + i + OFF; }
};
// Constants of the point update (Eqs. 19-23): ncoef = -lamdt / (2 h^2) scales the flux
// divergence of the scaled fluxes Phi = 2 h F; the relaxed diagonal is carried as
// den_c = (1 + alpha_c) / omega = kb + ka (S_a + S_b), ka = lamdt / (2 h^2 omega), kb = 1 / omega,
// where S_a = (eta_lo + eta) + (eta + eta_hi) is the sum of the cell's two face eta sums along
// axis a (alpha_c = lamdt / h^2 times the sum, over the axes a != c, of the mean face eta on both
// sides).  The host computes all three in float64 and rounds them once.
template <typename T>
struct RbK {
    T ncoef, ka, kb;
};
template <typename T>
RbK<T> rb_constants(double lamdt, double h, double omega) {
    const double coef = lamdt / (2.0 * h * h);
    return RbK<T>{(T)-coef, (T)(coef / omega), (T)(1.0 / omega)};
}

// Arithmetic of the point update, every operation rounded once (never contracted by the
// compiler), in float32 or float64.
__device__ __forceinline__ float v_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float v_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float v_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float v_mad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double v_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double v_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double v_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double v_mad(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename V>
__device__ __forceinline__ V v_splat(float x) {
    return V(x);
}
template <typename V>
__device__ __forceinline__ V v_zero() {
    return v_splat<V>(0.0f);
}

// The relaxed update ev + res / den: float32 through the hardware's approximate reciprocal
// (rcp.approx, relative error below 2^-23; a smoothing weight needs no correctly rounded
// quotient) and one FMA, float64 with an exact division.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rb_relax(float ev, float res, float den) { return v_mad(res, rcp_approx(den), ev); }
__device__ __forceinline__ double rb_relax(double ev, double res, double den) { return v_add(ev, __ddiv_rn(res, den)); }

// The point update of one colour pass (Eq. 19 with R from Eq. 20 and alpha from Eqs. 21-23),
// written against an accessor that returns component C of the field, or eta, at a compile-time
// offset (DX, DY, DZ) from the updated cell.  Every fused sweep kernel goes through these
// functions, whatever its staging: the rounding of each update is the same in all of them.
//
// face_pair: the divergence contribution of flux component C through the cell's two faces along
// axis AX, es_hi Q_hi - es_lo Q_lo with Phi = es Q, Q = T / 4 - N (Eqs. 9-10).  The tangential
// sums of the two faces (Eq. 10) share their middle difference, so they are formed as
//   T_hi = D(+AX) + D(0),  T_lo = D(0) + D(-AX),  D(s) = B_AX(s + e_C) - B_AX(s - e_C),
// the same four values each, regrouped (4 additions for both faces instead of 6).  The low face
// carries -Q (N - T/4, the same bits negated), so no operation needs a negated operand.
template <typename V, int AX, int C, class A>
__device__ __forceinline__ V face_pair(const A &a, V es_lo, V es_hi) {
    constexpr int AXX = AX == 0, AXY = AX == 1, AXZ = AX == 2;
    constexpr int CX = C == 0, CY = C == 1, CZ = C == 2;
    const V d0 = v_sub(a.template B<AX, CX, CY, CZ>(), a.template B<AX, -CX, -CY, -CZ>());
    const V dp = v_sub(a.template B<AX, AXX + CX, AXY + CY, AXZ + CZ>(), a.template B<AX, AXX - CX, AXY - CY, AXZ - CZ>());
    const V dm = v_sub(a.template B<AX, CX - AXX, CY - AXY, CZ - AXZ>(), a.template B<AX, -CX - AXX, -CY - AXY, -CZ - AXZ>());
    const V c0 = a.template B<C, 0, 0, 0>();
    const V q_hi = v_mad(v_add(dp, d0), v_splat<V>(0.25f), v_sub(c0, a.template B<C, AXX, AXY, AXZ>()));
    const V mq_lo = v_mad(v_add(d0, dm), v_splat<V>(-0.25f), v_sub(c0, a.template B<C, -AXX, -AXY, -AXZ>()));
    return v_mad(es_hi, q_hi, v_mul(es_lo, mq_lo));
}

// face sums of eta: eta_lo + eta on the low face, eta + eta_hi on the high face, along x, y, z
template <typename V, class A>
__device__ __forceinline__ void face_sums(const A &a, V es[6]) {
    const V e0 = a.template E<0, 0, 0>();
    es[0] = v_add(a.template E<-1, 0, 0>(), e0);
    es[1] = v_add(e0, a.template E<1, 0, 0>());
    es[2] = v_add(a.template E<0, -1, 0>(), e0);
    es[3] = v_add(e0, a.template E<0, 1, 0>());
    es[4] = v_add(a.template E<0, 0, -1>(), e0);
    es[5] = v_add(e0, a.template E<0, 0, 1>());
}

// the flux divergence of the cell (Eq. 8) from its face sums
template <typename V, class A>
__device__ __forceinline__ void cell_divergence(const A &a, const V es[6], V dv[3]) {
    dv[0] = v_add(face_pair<V, 1, 0>(a, es[2], es[3]), face_pair<V, 2, 0>(a, es[4], es[5]));
    dv[1] = v_add(face_pair<V, 0, 1>(a, es[0], es[1]), face_pair<V, 2, 1>(a, es[4], es[5]));
    dv[2] = v_add(face_pair<V, 0, 2>(a, es[0], es[1]), face_pair<V, 1, 2>(a, es[2], es[3]));
}

// face sums and den_c
template <typename V, class A>
__device__ __forceinline__ void rb_faces_den(const A &a, const RbK<V> &K, V es[6], V den[3]) {
    face_sums<V>(a, es);
    const V sx = v_add(es[0], es[1]), sy = v_add(es[2], es[3]), sz = v_add(es[4], es[5]);
    den[0] = v_mad(K.ka, v_add(sy, sz), K.kb);
    den[1] = v_mad(K.ka, v_add(sz, sx), K.kb);
    den[2] = v_mad(K.ka, v_add(sx, sy), K.kb);
}

template <typename V, class A>
__device__ __forceinline__ void rb_update_acc(const A &a, const RbK<V> &K, const V rr[3], V out[3]) {
    V es[6], den[3], dv[3];
    rb_faces_den<V>(a, K, es, den);
    cell_divergence<V>(a, es, dv);
    const V ev[3] = {a.template B<0, 0, 0, 0>(), a.template B<1, 0, 0, 0>(), a.template B<2, 0, 0, 0>()};
#pragma unroll
    for (int c = 0; c < 3; c++) out[c] = rb_relax(ev[c], v_mad(K.ncoef, dv[c], v_sub(rr[c], ev[c])), den[c]);
}

// The first sweep from e = 0, where the red colour pass reduces to e = r / den (every flux of the
// pre-pass state vanishes) and the black pass sees red values at the face neighbours of a black
// cell and zeros at its edge neighbours and at itself.  The two updates below are
// rb_update_acc with those zeros folded in: every dropped term is an exact +-0 there, so the
// results are the same bits (up to the sign of a zero).  The tangential difference of a black
// cell is the same for its two faces along an axis (D(+-AX) = 0), so a black update reads 31
// tile values instead of about 46.
template <typename V, class A>
__device__ __forceinline__ void red_from_zero_acc(const A &a, const RbK<V> &K, const V rr[3], V out[3]) {
    V es[6], den[3];
    rb_faces_den<V>(a, K, es, den);
#pragma unroll
    for (int c = 0; c < 3; c++) out[c] = rb_relax(v_zero<V>(), rr[c], den[c]);
}

template <typename V, int AX, int C, class A>
__device__ __forceinline__ V face_pair_zero(const A &a, V es_lo, V es_hi) {
    constexpr int AXX = AX == 0, AXY = AX == 1, AXZ = AX == 2;
    constexpr int CX = C == 0, CY = C == 1, CZ = C == 2;
    const V d0 = v_sub(a.template B<AX, CX, CY, CZ>(), a.template B<AX, -CX, -CY, -CZ>());
    const V q_hi = v_sub(v_mul(d0, v_splat<V>(0.25f)), a.template B<C, AXX, AXY, AXZ>());
    const V mq_lo = v_sub(v_mul(d0, v_splat<V>(-0.25f)), a.template B<C, -AXX, -AXY, -AXZ>());
    return v_mad(es_hi, q_hi, v_mul(es_lo, mq_lo));
}

template <typename V, class A>
__device__ __forceinline__ void black_after_zero_acc(const A &a, const RbK<V> &K, const V rr[3], V out[3]) {
    V es[6], den[3];
    rb_faces_den<V>(a, K, es, den);
    const V dv[3] = {v_add(face_pair_zero<V, 1, 0>(a, es[2], es[3]), face_pair_zero<V, 2, 0>(a, es[4], es[5])),
                     v_add(face_pair_zero<V, 0, 1>(a, es[0], es[1]), face_pair_zero<V, 2, 1>(a, es[4], es[5])),
                     v_add(face_pair_zero<V, 0, 2>(a, es[0], es[1]), face_pair_zero<V, 1, 2>(a, es[2], es[3]))};
#pragma unroll
    for (int c = 0; c < 3; c++) out[c] = rb_relax(v_zero<V>(), v_mad(K.ncoef, dv[c], rr[c]), den[c]);
}

// accessor of a staged tile (geometry G: rows RRS apart, planes PS, components CS)
template <typename T, typename G>
struct TileAcc {
    const T *tB, *tE;
    int p;
    template <int C, int DX, int DY, int DZ>
    __device__ __forceinline__ T B() const {
        return tB[C * G::CS + p + DX + DY * G::RRS + DZ * G::PS];
    }
    template <int DX, int DY, int DZ>
    __device__ __forceinline__ T E() const {
        return tE[p + DX + DY * G::RRS + DZ * G::PS];
    }
};

template <typename T, typename G = G12<T>>
__device__ __forceinline__ void rb_update(const T *__restrict__ tB, const T *__restrict__ tE, int p, const RbK<T> &K,
                                          const T rr[3], T out[3]) {
    rb_update_acc<T>(TileAcc<T, G>{tB, tE, p}, K, rr, out);
}

template <typename T>
__global__ void __launch_bounds__(256) k_smooth_rb(GridDev g, const T *__restrict__ e_in, T *__restrict__ e_out,
                                                   const T *__restrict__ r, const T *__restrict__ eta, RbK<T> K) {
    using G = G12<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tB = reinterpret_cast<T *>(smem_raw);  // [3][12 planes][12 rows][RRS]
    T *tE = tB + 3 * G::CS;
    __shared__ int snb[27];
    const int b = blockIdx.x;
    if (skip_block(g, b)) return;
    stage_nbr(snb, g.nbr, b);
    __syncthreads();
    stage_rows<T, 3, 2, G::RRS, G::OFF>(tB, e_in, snb, nullptr);
    stage_rows<T, 1, 2, G::RRS, G::OFF>(tE, eta, snb, nullptr);
    __syncthreads();
    // Red cells ((i+j+k) even): the block's 256, one per thread in the same pattern as the black
    // phase (a warp reads 8 rows x 4 cells of one plane: distinct banks), then the 240 of the
    // ring (faces and edges of the 10^3 box, corners excluded), one per thread t < 240:
    // t < 192: face slab f = t/32 (axis f/2 at -1 or 8), 8 lines x 4 red cells;
    // t >= 192: edge e = (t-192)/4 (two axes out), 4 red cells along the third axis.
    T nv[2][3];
    int np[2];
#pragma unroll
    for (int s4 = 0; s4 < 2; s4++) {
        np[s4] = -1;
        const int t = threadIdx.x;
        int li, lj, lk;
        if (s4 == 0) {
            lk = t >> 5;
            lj = (t >> 2) & 7;
            li = 2 * (t & 3) + ((lj + lk) & 1);
        } else {
            if (t >= 240) continue;
            int c[3];
            if (t < 192) {
                const int f = t >> 5, ax = f >> 1, q = t & 31;
                const int v = q >> 2, u2 = q & 3;
                const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
                c[ax] = (f & 1) ? 8 : -1;
                c[a2] = v;
                c[a1] = 2 * u2 + ((c[ax] + v) & 1);
            } else {
                const int e = (t - 192) >> 2, w2 = (t - 192) & 3;
                const int pr = e >> 2, sg = e & 3;  // axis pair (0,1), (0,2), (1,2) and its sign combination
                const int a1 = pr == 2 ? 1 : 0, a2 = pr == 0 ? 1 : 2, af = 3 - a1 - a2;
                c[a1] = (sg & 1) ? 8 : -1;
                c[a2] = (sg & 2) ? 8 : -1;
                c[af] = 2 * w2 + ((c[a1] + c[a2]) & 1);
            }
            li = c[0];
            lj = c[1];
            lk = c[2];
        }
        const int di = li < 0 ? -1 : (li > 7 ? 1 : 0), dj = lj < 0 ? -1 : (lj > 7 ? 1 : 0), dk = lk < 0 ? -1 : (lk > 7 ? 1 : 0);
        const int src = snb[(dk + 1) * 9 + (dj + 1) * 3 + (di + 1)];
        const int off = ((lk - 8 * dk) * 8 + (lj - 8 * dj)) * 8 + (li - 8 * di);
        const T rr[3] = {r[(size_t)src * 3 * B3 + off], r[(size_t)src * 3 * B3 + B3 + off], r[(size_t)src * 3 * B3 + 2 * B3 + off]};
        np[s4] = G::at(li + 2, lj + 2, lk + 2);
        rb_update(tB, tE, np[s4], K, rr, nv[s4]);
    }
    __syncthreads();
#pragma unroll
    for (int s4 = 0; s4 < 2; s4++)
        if (np[s4] >= 0)
            for (int c = 0; c < 3; c++) tB[c * G::CS + np[s4]] = nv[s4][c];
    __syncthreads();
    // black cells of the block, one per thread, then the whole block is written out
    const int t = threadIdx.x;
    const int k = t >> 5, j = (t >> 2) & 7;
    const int ib = 2 * (t & 3) + ((j + k + 1) & 1), ir = 2 * (t & 3) + ((j + k) & 1);
    const int cb = (k * 8 + j) * 8 + ib, cr = (k * 8 + j) * 8 + ir;
    const T rr[3] = {r[(size_t)b * 3 * B3 + cb], r[(size_t)b * 3 * B3 + B3 + cb], r[(size_t)b * 3 * B3 + 2 * B3 + cb]};
    T out[3];
    const int pb = G::at(ib + 2, j + 2, k + 2), pr = G::at(ir + 2, j + 2, k + 2);
    rb_update(tB, tE, pb, K, rr, out);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        e_out[((size_t)b * 3 + c) * B3 + cb] = out[c];
        e_out[((size_t)b * 3 + c) * B3 + cr] = tB[c * G::CS + pr];
    }
}

template <typename T>
cudaError_t launch_smooth_rb(const GridDev &g, const T *e_in, T *e_out, const T *r, const T *eta, double lamdt,
                             cudaStream_t s) {
    if (g.nblk == 0) return cudaSuccess;
    const size_t sm = 4 * G12<T>::CS * sizeof(T);
    // set once per process (thread-safe static initialisation)
    static const bool attr = (cudaFuncSetAttribute(k_smooth_rb<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm), true);
    (void)attr;
    k_smooth_rb<T><<<g.nblk, 256, sm, s>>>(g, e_in, e_out, r, eta, rb_constants<T>(lamdt, g.h, g.omega));
    return cudaGetLastError();
}
template cudaError_t launch_smooth_rb<float>(const GridDev &, const float *, float *, const float *, const float *, double,
                                             cudaStream_t);
template cudaError_t launch_smooth_rb<double>(const GridDev &, const double *, double *, const double *, const double *,
                                              double, cudaStream_t);

// ------------------------------------------------------------------ fused sweep on brick pairs
// The fused sweep above for two x-adjacent blocks A = 2q and B = 2q + 1 per thread block (512
// threads): a 20 x 12 x 12 tile (two-cell halo) shares its halo and ring between the two
// blocks, so per block it stages 17% fewer values and recomputes 20% fewer ring updates.
// Rows are 24 floats apart: the warp pattern of the brick's same-colour cells (4 rows x 8
// cells at stride 2) then falls on 32 distinct banks; each tile row starts on a 16-byte
// boundary and is staged as five 16-byte words.  Used for float32 grids whose every block pair (2q, 2q+1)
// is x-adjacent and whose blocks all have their 26 neighbours.  Bounded to 40 registers so
// that 3 thread blocks (48 warps) share an SM.  Measured per 256^3 sweep: 0.362 ms; 0.401 ms
// before the staging stores and the ring order were arranged by bank (conflicts 3.8 M -> 0.8 M
// per 128^3 sweep); 0.427 ms at 54 registers (2 per SM); 0.431 ms for the one-block kernel.
struct G20 {
    static constexpr int SX = 20, S = 12, RRS = 24, PS = S * RRS + 4, CS = S * PS, OFF = 0;
    __device__ static __forceinline__ int at(int i, int j, int k) { return k * PS + j * RRS + i + OFF; }
};

// red cells of the brick's one-cell ring (faces and edges, no corners): 384 entries
// (li+1) | (lj+1) << 5 | (lk+1) << 10, li in [-1, 16], lj, lk in [-1, 8], ordered for the 12
// warps that update them so that shared-memory banks (tile offset mod 32) repeat little within a
// warp: with the strides of G20 a bank holds at most 17 of the 384 cells and at least 8, so 7
// warps take one cell per bank and 5 warps at most two.  Built at compile time.
struct Ring2 {
    uint32_t v[384];
};
constexpr int ring2_bank(int i, int j, int k) { return ((i + 2 + G20::OFF) + (j + 2) * G20::RRS + (k + 2) * G20::PS) & 31; }
constexpr bool ring2_cell(int i, int j, int k) {
    const int out = (i < 0 || i > 15) + (j < 0 || j > 7) + (k < 0 || k > 7);
    return out != 0 && out != 3 && ((i + j + k) & 1) == 0;
}
constexpr Ring2 make_ring2() {
    Ring2 m{};
    int cnt[32] = {};
    for (int k = -1; k <= 8; k++)
        for (int j = -1; j <= 8; j++)
            for (int i = -1; i <= 16; i++)
                if (ring2_cell(i, j, k)) cnt[ring2_bank(i, j, k)]++;
    int maxc = 0;
    for (int r = 0; r < 32; r++) maxc = cnt[r] > maxc ? cnt[r] : maxc;
    const int A = 24 - maxc < 12 ? 24 - maxc : 12;  // warps with one cell per bank
    int fill[12] = {}, seen[32] = {}, two[12][32] = {};
    for (int k = -1; k <= 8; k++)
        for (int j = -1; j <= 8; j++)
            for (int i = -1; i <= 16; i++) {
                if (!ring2_cell(i, j, k)) continue;
                const int r = ring2_bank(i, j, k), n = seen[r]++;
                int w = n;
                if (n >= A) {
                    w = -1;
                    for (int c = A; c < 12; c++)
                        if (two[c][r] < 2 && fill[c] < 32 && (w < 0 || fill[c] < fill[w])) w = c;
                    two[w][r]++;
                }
                m.v[w * 32 + fill[w]++] = (uint32_t)(i + 1) | ((uint32_t)(j + 1) << 5) | ((uint32_t)(k + 1) << 10);
            }
    return m;
}
__device__ const Ring2 g_ring2 = make_ring2();

// ZERO: the sweep starts from e = 0 (the first pre-smoothing sweep of a level): e_in is not read,
// only eta is staged, the red pass is pointwise and the black pass reads only red values.
template <bool ZERO>
__global__ void __launch_bounds__(512, 3) k_smooth_rb2(GridDev g, const float *__restrict__ e_in, float *__restrict__ e_out,
                                                    const float *__restrict__ r, const float *__restrict__ eta,
                                                    RbK<float> K) {
    using G = G20;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tB = reinterpret_cast<float *>(smem_raw);  // [3][12 planes][12 rows][RRS]
    float *tE = tB + 3 * G::CS;
    // neighbourhood of the brick: block columns bx = -1, 0 (A), 1 (B), 2 along x, by dj, dk
    __shared__ int snb[36];
    const int A = 2 * blockIdx.x;
    if (skip_block(g, A)) return;
    if (threadIdx.x < 36) {
        const int bx = threadIdx.x % 4 - 1, dj = (threadIdx.x / 4) % 3 - 1, dk = threadIdx.x / 12 - 1;
        const int base = bx <= 1 ? A : A + 1, dx = bx <= 1 ? bx : 1;
        snb[threadIdx.x] = __ldg(g.nbr + base * 27 + (dk + 1) * 9 + (dj + 1) * 3 + (dx + 1));
    }
    __syncthreads();
    // one task per (field component, tile row): the 20 values of the row (halo pair, 8 + 8
    // interior cells, halo pair) as five 16-byte stores; each quarter-warp takes 4 rows of 2
    // consecutive planes, whose 16-byte bank groups are distinct (plane stride = 4 mod 32)
    // from e = 0 only eta is staged (e is never read before the red values are written)
    for (int task = ZERO ? 3 * 144 + threadIdx.x : threadIdx.x; task < 4 * 144; task += blockDim.x) {
        const int c = task / 144, u = task - c * 144;
        const int q = u >> 3, w = u & 7;
        const int tk = 2 * (q / 3) + (w >> 2), tj = 4 * (q % 3) + (w & 3);
        const int lj = tj - 2, lk = tk - 2;
        const int dj = lj < 0 ? -1 : (lj > 7 ? 1 : 0), dk = lk < 0 ? -1 : (lk > 7 ? 1 : 0);
        const int rowoff = ((lk - 8 * dk) * 8 + (lj - 8 * dj)) * 8;
        const int *nb = snb + (dk + 1) * 12 + (dj + 1) * 4;
        const float *F = c < 3 ? e_in : eta;
        const int nc = c < 3 ? 3 : 1, cc = c < 3 ? c : 0;
        float4 *dst = reinterpret_cast<float4 *>((c < 3 ? tB + c * G::CS : tE) + tk * G::PS + tj * G::RRS + G::OFF);
        const float2 lo = __ldg(reinterpret_cast<const float2 *>(F + ((size_t)nb[0] * nc + cc) * B3 + rowoff + 6));
        const float4 *pa = reinterpret_cast<const float4 *>(F + ((size_t)nb[1] * nc + cc) * B3 + rowoff);
        const float4 *pb = reinterpret_cast<const float4 *>(F + ((size_t)nb[2] * nc + cc) * B3 + rowoff);
        const float2 hi = __ldg(reinterpret_cast<const float2 *>(F + ((size_t)nb[3] * nc + cc) * B3 + rowoff));
        const float4 a0 = __ldg(pa), a1 = __ldg(pa + 1), b0 = __ldg(pb), b1 = __ldg(pb + 1);
        dst[0] = make_float4(lo.x, lo.y, a0.x, a0.y);
        dst[1] = make_float4(a0.z, a0.w, a1.x, a1.y);
        dst[2] = make_float4(a1.z, a1.w, b0.x, b0.y);
        dst[3] = make_float4(b0.z, b0.w, b1.x, b1.y);
        dst[4] = make_float4(b1.z, b1.w, hi.x, hi.y);
    }
    const int t = threadIdx.x;
    const int k = t >> 6, j = (t >> 3) & 7, i2 = t & 7;
    const int ir = 2 * i2 + ((j + k) & 1), ib = 2 * i2 + ((j + k + 1) & 1);  // both in block A (i2 < 4) or B
    const int own = A + (i2 >> 2);
    // the red and the black cell of a thread are the x-pair (2 i2, 2 i2 + 1) of a block row:
    // their right-hand sides come in, and their results go out, as one 8-byte word each
    const int cpair = (k * 8 + j) * 8 + ((2 * i2) & 7);
    const bool red_even = ((j + k) & 1) == 0;
    float rr0[3], rr1[3] = {0.f, 0.f, 0.f}, rrb[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float2 v = *reinterpret_cast<const float2 *>(r + ((size_t)own * 3 + c) * B3 + cpair);
        rr0[c] = red_even ? v.x : v.y;
        rrb[c] = red_even ? v.y : v.x;
    }
    int p1 = -1;
    if (t < 384) {
        const uint32_t code = __ldg(&g_ring2.v[t]);
        const int li = (int)(code & 31u) - 1, lj = (int)((code >> 5) & 31u) - 1, lk = (int)((code >> 10) & 31u) - 1;
        const int bx = li < 0 ? -1 : (li > 15 ? 2 : (li >> 3));
        const int dj = lj < 0 ? -1 : (lj > 7 ? 1 : 0), dk = lk < 0 ? -1 : (lk > 7 ? 1 : 0);
        const int src = snb[(dk + 1) * 12 + (dj + 1) * 4 + (bx + 1)];
        const int off = ((lk - 8 * dk) * 8 + (lj - 8 * dj)) * 8 + (li - 8 * bx);
#pragma unroll
        for (int c = 0; c < 3; c++) rr1[c] = r[((size_t)src * 3 + c) * B3 + off];
        p1 = G::at(li + 2, lj + 2, lk + 2);
    }
    __syncthreads();
    // red: the brick's 512 (one per thread), then the 384 of its ring, from the pre-sweep state
    float nv0[3], nv1[3];
    const int p0 = G::at(ir + 2, j + 2, k + 2);
    if constexpr (ZERO) {  // nothing of e is read: no barrier before the red values are stored
        red_from_zero_acc<float>(TileAcc<float, G>{tB, tE, p0}, K, rr0, nv0);
        if (p1 >= 0) red_from_zero_acc<float>(TileAcc<float, G>{tB, tE, p1}, K, rr1, nv1);
    } else {
        rb_update<float, G>(tB, tE, p0, K, rr0, nv0);
        if (p1 >= 0) rb_update<float, G>(tB, tE, p1, K, rr1, nv1);
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
        tB[c * G::CS + p0] = nv0[c];
        if (p1 >= 0) tB[c * G::CS + p1] = nv1[c];
    }
    __syncthreads();
    // black cells of the brick from the post-red state, then both blocks are written out
    float out[3];
    if constexpr (ZERO)  // black cells read only red neighbours (their black neighbours are 0)
        black_after_zero_acc<float>(TileAcc<float, G>{tB, tE, G::at(ib + 2, j + 2, k + 2)}, K, rrb, out);
    else
        rb_update<float, G>(tB, tE, G::at(ib + 2, j + 2, k + 2), K, rrb, out);
#pragma unroll
    for (int c = 0; c < 3; c++)
        *reinterpret_cast<float2 *>(e_out + ((size_t)own * 3 + c) * B3 + cpair) =
            red_even ? make_float2(nv0[c], out[c]) : make_float2(out[c], nv0[c]);
}

cudaError_t launch_smooth_rb2(const GridDev &g, const float *e_in, float *e_out, const float *r, const float *eta,
                              double lamdt, cudaStream_t s) {
    if (g.nblk == 0) return cudaSuccess;
    const size_t sm = 4 * G20::CS * sizeof(float);
    static const bool attr = (cudaFuncSetAttribute(k_smooth_rb2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                              cudaFuncSetAttribute(k_smooth_rb2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                              true);
    (void)attr;
    const RbK<float> K = rb_constants<float>(lamdt, g.h, g.omega);
    if (e_in)
        k_smooth_rb2<false><<<g.nblk / 2, 512, sm, s>>>(g, e_in, e_out, r, eta, K);
    else  // from e = 0
        k_smooth_rb2<true><<<g.nblk / 2, 512, sm, s>>>(g, nullptr, e_out, r, eta, K);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ residual on brick pairs
// The float32 operator and residual of the inner solve on the same x-adjacent block pairs as
// the pair sweep (512 threads, one thread block per pair), with the flux divergence formed per
// cell by the sweep's face_pair (Eqs. 8-10) instead of through face-flux arrays: no flux
// arrays, one barrier, a 18 x 10 x 10 tile (one-cell halo; rows staged as 16-byte words with
// the block interiors 16-byte aligned at OFF = 3).  Modes:
//   APPLY:    out = X + kc divF(X)                    (L X, the Krylov operator)
//   residual: out = (Y - X) + kc divF(X), kc = -lamdt / (2 h^2)   (Eq. 20)
// and RESTRICT: the residual's octet means written into the coarser grid (Sec. 2.2), for grids
// whose children sit in Morton octets (block b's parent is b / 8, its octant b % 8).  A warp
// takes 8 cells of a row x 2 rows x 2 planes of one block: every 2^3 octet is in one warp (sums
// by three shuffles), and with rows 24 and planes 240 floats apart (240 = 16 mod 32) its
// shared-memory reads at one offset fall on 32 distinct banks.
struct G18 {
    static constexpr int S = 10, RRS = 24, PS = S * RRS, CS = S * PS, OFF = 3;
    __device__ static __forceinline__ int at(int i, int j, int k) { return k * PS + j * RRS + i + OFF; }
};

// Contribution of a cell's face along AX to the flux divergence of component C, for the face on
// side so (+-1 cell along AX, as a tile offset) with qs = +-1/4: es Q on the high side, -es Q on
// the low one -- the terms of face_pair for that face alone, in the same operations.
template <int AX, int C>
__device__ __forceinline__ float octet_face(const float *__restrict__ tB, int p, int so, float qs, float es) {
    constexpr int SC = C == 0 ? 1 : (C == 1 ? G18::RRS : G18::PS);
    const float *BA = tB + AX * G18::CS + p, *BC = tB + C * G18::CS + p;
    const float d0 = v_sub(BA[SC], BA[-SC]);
    const float dn = v_sub(BA[so + SC], BA[so - SC]);
    return v_mul(es, v_mad(v_add(dn, d0), qs, v_sub(BC[0], BC[so])));
}

// NV >= 0 (APPLY only): also the FGMRES products of the output w with the NV vectors of V and
// with itself, <w, v_i> and <w, w>, each weighted by wt (h^3 for the cells of a single-level
// grid) and folded per block pair in a fixed order into part[i][pair] (column-major, so that
// the column sums read contiguous rows).
// OCT (residual + restriction with no fine output): the restriction needs only the octet sums
// of the flux divergence, and in the conservative form (Eq. 8) every flux through a face inside
// an octet enters its two cells with opposite signs, so the sum over the octet is the net flux
// through the octet's 24 outer faces.  Each cell of an octet sits at one of its corners and
// owns exactly one outer face per axis (the high face where its coordinate is odd, the low one
// where it is even); it computes those three faces instead of its six, and the octet sum of
// (Y - X) + kc divF(X) is formed as before.  Equal to the full form in exact arithmetic (the
// internal fluxes cancel); about 40% fewer operations and 30% fewer tile reads per cell.
template <bool APPLY, bool RESTRICT, int NV = -1, bool OCT = false>
__global__ void __launch_bounds__(512, NV >= 0 ? 3 : 4)
    k_pair_op(GridDev g, const float *__restrict__ X, const float *__restrict__ Y, const float *__restrict__ eta, float kc,
              float *__restrict__ out, float *__restrict__ coarse, VecSet V = VecSet(), double wt = 0.0,
              double *__restrict__ part = nullptr) {
    using G = G18;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tB = reinterpret_cast<float *>(smem_raw);  // [3][10 planes][10 rows][RRS]
    float *tE = tB + 3 * G::CS;
    __shared__ int snb[36];
    const int A = 2 * blockIdx.x;
    if (skip_block(g, A)) return;
    if (threadIdx.x < 36) {
        const int bx = threadIdx.x % 4 - 1, dj = (threadIdx.x / 4) % 3 - 1, dk = threadIdx.x / 12 - 1;
        const int base = bx <= 1 ? A : A + 1, dx = bx <= 1 ? bx : 1;
        snb[threadIdx.x] = __ldg(g.nbr + base * 27 + (dk + 1) * 9 + (dj + 1) * 3 + (dx + 1));
    }
    __syncthreads();
    // one task per (field component, tile row): 1 + 8 + 8 + 1 values, the interiors as 16-byte words
    if (threadIdx.x < 400) {
        const int c = threadIdx.x / 100, u = threadIdx.x - c * 100;
        const int tk = u / 10, tj = u - 10 * tk;
        const int lj = tj - 1, lk = tk - 1;
        const int dj = lj < 0 ? -1 : (lj > 7 ? 1 : 0), dk = lk < 0 ? -1 : (lk > 7 ? 1 : 0);
        const int rowoff = ((lk - 8 * dk) * 8 + (lj - 8 * dj)) * 8;
        const int *nb = snb + (dk + 1) * 12 + (dj + 1) * 4;
        const float *F = c < 3 ? X : eta;
        const int nc = c < 3 ? 3 : 1, cc = c < 3 ? c : 0;
        float *row = (c < 3 ? tB + c * G::CS : tE) + tk * G::PS + tj * G::RRS + G::OFF;
        const float lo = __ldg(F + ((size_t)nb[0] * nc + cc) * B3 + rowoff + 7);
        const float4 *pa = reinterpret_cast<const float4 *>(F + ((size_t)nb[1] * nc + cc) * B3 + rowoff);
        const float4 *pb = reinterpret_cast<const float4 *>(F + ((size_t)nb[2] * nc + cc) * B3 + rowoff);
        const float hi = __ldg(F + ((size_t)nb[3] * nc + cc) * B3 + rowoff);
        const float4 a0 = __ldg(pa), a1 = __ldg(pa + 1), b0 = __ldg(pb), b1 = __ldg(pb + 1);
        row[0] = lo;
        float4 *r4 = reinterpret_cast<float4 *>(row + 1);
        r4[0] = a0;
        r4[1] = a1;
        r4[2] = b0;
        r4[3] = b1;
        row[17] = hi;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = lane & 7, y = 2 * (w & 3) + ((lane >> 3) & 1), z = 2 * ((w >> 2) & 3) + (lane >> 4);
    const int cell = (z * 8 + y) * 8 + x;
    constexpr int ND = NV >= 0 ? NV + 1 : 1;
    float dots[ND];
#pragma unroll
    for (int i = 0; i < ND; i++) dots[i] = 0.f;
#pragma unroll
    for (int h = 0; h < 2; h++) {  // the same cell of block A, then of block B
        const int b = A + h;
        const TileAcc<float, G> acc{tB, tE, G::at(1 + 8 * h + x, 1 + y, 1 + z)};
        float dv[3];
        if constexpr (OCT) {
            const int p = acc.p, ox = (x & 1) ? 1 : -1, oy = (y & 1) ? G::RRS : -G::RRS, oz = (z & 1) ? G::PS : -G::PS;
            const float qx = (x & 1) ? 0.25f : -0.25f, qy = (y & 1) ? 0.25f : -0.25f, qz = (z & 1) ? 0.25f : -0.25f;
            const float e0 = tE[p];
            const float esx = v_add(e0, tE[p + ox]), esy = v_add(e0, tE[p + oy]), esz = v_add(e0, tE[p + oz]);
            dv[0] = v_add(octet_face<1, 0>(tB, p, oy, qy, esy), octet_face<2, 0>(tB, p, oz, qz, esz));
            dv[1] = v_add(octet_face<0, 1>(tB, p, ox, qx, esx), octet_face<2, 1>(tB, p, oz, qz, esz));
            dv[2] = v_add(octet_face<0, 2>(tB, p, ox, qx, esx), octet_face<1, 2>(tB, p, oy, qy, esy));
        } else {
            float es[6];
            face_sums<float>(acc, es);
            cell_divergence<float>(acc, es, dv);
        }
        const float ev[3] = {acc.template B<0, 0, 0, 0>(), acc.template B<1, 0, 0, 0>(), acc.template B<2, 0, 0, 0>()};
        float o[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const size_t id = ((size_t)b * 3 + c) * B3 + cell;
            o[c] = v_mad(kc, dv[c], APPLY ? ev[c] : v_sub(Y[id], ev[c]));
            if (!OCT && out) out[id] = o[c];
            if constexpr (NV >= 0) {
#pragma unroll
                for (int i = 0; i < NV; i++) dots[i] = fmaf(o[c], __ldg(V.v[i] + id), dots[i]);
                dots[NV] = fmaf(o[c], o[c], dots[NV]);
            }
        }
        if constexpr (RESTRICT) {
            const int oct = b & 7, pb = b >> 3;
            const int cx = 4 * (oct & 1) + (x >> 1), cy = 4 * ((oct >> 1) & 1) + (y >> 1), cz = 4 * (oct >> 2) + (z >> 1);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                float sum = v_add(o[c], __shfl_xor_sync(0xffffffffu, o[c], 1));
                sum = v_add(sum, __shfl_xor_sync(0xffffffffu, sum, 8));
                sum = v_add(sum, __shfl_xor_sync(0xffffffffu, sum, 16));
                if ((lane & 0x19) == 0) coarse[((size_t)pb * 3 + c) * B3 + (cz * 8 + cy) * 8 + cx] = v_mul(sum, 0.125f);
            }
        }
    }
    if constexpr (NV >= 0) {  // warp sums, then the 16 warps in order (the tile is free by now)
        __syncthreads();
        double *sred = reinterpret_cast<double *>(smem_raw);  // [16][NV + 1]
#pragma unroll
        for (int i = 0; i <= NV; i++) {
            float v = dots[i];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sred[w * (NV + 1) + i] = (double)v;
        }
        __syncthreads();
        if (threadIdx.x <= NV) {
            double a = 0.0;
            for (int q = 0; q < 16; q++) a += sred[q * (NV + 1) + threadIdx.x];
            part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = a * wt;
        }
    }
}

cudaError_t launch_pair_op(const GridDev &g, const float *X, const float *Y, const float *eta, double kc, bool apply,
                           float *out, float *coarse, cudaStream_t s) {
    if (g.nblk == 0) return cudaSuccess;
    const size_t sm = 4 * G18::CS * sizeof(float);
    static const bool attr = (cudaFuncSetAttribute(k_pair_op<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                              cudaFuncSetAttribute(k_pair_op<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                              cudaFuncSetAttribute(k_pair_op<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                              cudaFuncSetAttribute(k_pair_op<false, true, -1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                              true);
    (void)attr;
    if (apply)
        k_pair_op<true, false><<<g.nblk / 2, 512, sm, s>>>(g, X, nullptr, eta, (float)kc, out, nullptr);
    else if (coarse && !out)  // only the octet means: outer faces of each octet
        k_pair_op<false, true, -1, true><<<g.nblk / 2, 512, sm, s>>>(g, X, Y, eta, (float)kc, nullptr, coarse);
    else if (coarse)
        k_pair_op<false, true><<<g.nblk / 2, 512, sm, s>>>(g, X, Y, eta, (float)kc, out, coarse);
    else
        k_pair_op<false, false><<<g.nblk / 2, 512, sm, s>>>(g, X, Y, eta, (float)kc, out, nullptr);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FGMRES scalars
// One thread per instance: the steps of FGMRES(m) (Saad 1993) that the single-problem solver
// takes on the host, in the same order and float64 arithmetic, for every instance of a batch.
__global__ void __launch_bounds__(128) k_fg(FgState f, int op, int j) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= f.K) return;
    constexpr int KC = KMAX + 1;
    const double *d = f.dots + (size_t)q * KC;
    float *c = f.coef + (size_t)q * KC;
    double *H = f.Hm + (size_t)q * KC * KMAX, *cs = f.cs + (size_t)q * KMAX, *sn = f.sn + (size_t)q * KMAX;
    double *g = f.g + (size_t)q * KC;
    auto h = [&](int i, int k) -> double & { return H[i * KMAX + k]; };
    auto clear = [&](float scale) {
        for (int i = 0; i < KMAX; i++) c[i] = 0.f;
        c[KMAX] = scale;
    };
    switch (op) {
        case FG_START: {  // v_0 = rhs / beta0 for the instances that iterate
            const double b = sqrt(fmax(d[0], 0.0));
            f.beta0[q] = f.beta[q] = f.brest[q] = b;
            f.live[q] = f.run[q] && b > 0 && isfinite(b);
            clear(f.live[q] ? (float)(1.0 / b) : 1.f);
            break;
        }
        case FG_CYCLE: {  // a restart cycle begins: g = beta e_0
            f.arn[q] = f.live[q];
            f.jend[q] = 0;
            for (int i = 0; i < KC; i++) g[i] = 0.0;
            g[0] = f.beta[q];
            break;
        }
        case FG_ACT: {  // instances that take Arnoldi step j (their V-cycle is counted)
            if (q == 0) *f.any_need2 = 0;
            const uint8_t a = f.arn[q] && f.cycles[q] < f.max_outer;
            f.act[q] = a;
            f.imask[q] = a;
            f.cycles[q] += a;
            break;
        }
        case FG_ORTHO: {  // h_ij = <w, v_i>; one-pass normalisation unless cancellation is large
            clear(1.f);
            f.need2[q] = 0;
            if (!f.act[q]) break;
            double proj = 0.0;
            for (int i = 0; i <= j; i++) {
                h(i, j) = d[i];
                c[i] = (float)d[i];
                proj += d[i] * d[i];
            }
            const double ww = d[j + 1];
            if (ww - proj > 0.01 * ww) {
                f.hn[q] = sqrt(ww - proj);
                c[KMAX] = (float)(1.0 / f.hn[q]);
            } else {
                f.need2[q] = 1;
                atomicOr(f.any_need2, 1);  // the norm pass after orthogonalising runs
            }
            break;
        }
        case FG_RENORM: {  // the norm measured after orthogonalising, where the one pass was refused
            clear(1.f);
            if (!f.act[q] || !f.need2[q]) break;
            f.hn[q] = sqrt(fmax(d[0], 0.0));
            if (f.hn[q] > 0) c[KMAX] = (float)(1.0 / f.hn[q]);
            break;
        }
        case FG_GIVENS: {
            if (!f.act[q]) break;
            const double hnq = f.hn[q];
            h(j + 1, j) = hnq;
            for (int i = 0; i < j; i++) {
                const double t = cs[i] * h(i, j) + sn[i] * h(i + 1, j);
                h(i + 1, j) = -sn[i] * h(i, j) + cs[i] * h(i + 1, j);
                h(i, j) = t;
            }
            const double den = hypot(h(j, j), h(j + 1, j));
            cs[j] = den > 0 ? h(j, j) / den : 1.0;
            sn[j] = den > 0 ? h(j + 1, j) / den : 0.0;
            h(j, j) = den;
            h(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            f.jend[q] = j + 1;
            if (fabs(g[j + 1]) <= f.target[q] * f.beta0[q] || !(hnq > 0)) {
                f.arn[q] = 0;
                f.live[q] = 0;  // converged (or breakdown): no restart
            }
            break;
        }
        case FG_SOLVE: {  // x += sum y_i z_i with R y = g
            clear(1.f);
            const int je = f.jend[q];
            double y[KMAX];
            for (int i = je - 1; i >= 0; i--) {
                double t = g[i];
                for (int k = i + 1; k < je; k++) t -= h(i, k) * y[k];
                y[i] = h(i, i) != 0 ? t / h(i, i) : 0.0;
            }
            for (int i = 0; i < je; i++) c[i] = (float)(-y[i]);
            break;
        }
        case FG_RESTART_MASK: {  // restart where the instance is live and may take more cycles
            if (f.live[q] && (f.cycles[q] >= f.max_outer || f.jend[q] == 0)) f.live[q] = 0;
            f.imask[q] = f.live[q];
            break;
        }
        case FG_RESTART: {  // stop at the target, on breakdown, or when the cycle gained < 2x
            clear(1.f);
            if (!f.live[q]) break;
            const double b = sqrt(fmax(d[0], 0.0));
            f.beta[q] = b;
            if (b <= f.target[q] * f.beta0[q] || !(b > 0) || b > 0.5 * f.brest[q]) {
                f.live[q] = 0;
                break;
            }
            f.brest[q] = b;
            c[KMAX] = (float)(1.0 / b);
            break;
        }
    }
}

cudaError_t launch_fg(const FgState &f, FgOp op, int j, cudaStream_t s) {
    if (f.K == 0) return cudaSuccess;
    k_fg<<<(f.K + 127) / 128, 128, 0, s>>>(f, (int)op, j);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ inverse diagonal
// inv_c = omega / (1 + alpha_c), alpha_c = lamdt/h^2 sum_{a != c} (eta_{-1/2} + eta_{+1/2})
// with face eta the mean of the two cells (Eqs. 11, 21-23).
template <typename T>
__global__ void __launch_bounds__(512) k_invdiag(GridDev g, const T *__restrict__ eta, const T *__restrict__ Geta,
                                                 double lh2, T *__restrict__ inv) {
    using G = Geo<T>;
    __shared__ __align__(16) T tE[G::CS];
    __shared__ int snb[27];
    const int b = blockIdx.x;
    if (skip_block(g, b)) return;
    const int slot = g.gslot ? g.gslot[b] : -1;
    stage_nbr(snb, g.nbr, b);
    __syncthreads();
    stage_rows<T, 1, 1, G::RS, G::OFF>(tE, eta, snb, slot >= 0 && Geta ? Geta + (size_t)slot * T3 : nullptr);
    __syncthreads();
    // computed in T: the inverse diagonal only scales smoother updates
    const int t = threadIdx.x, i = t & 7, j = (t >> 3) & 7, k = t >> 6;
    const int p = G::at(i + 1, j + 1, k + 1);
    const T e0 = tE[p], h = T(0.5), l = (T)lh2;
    const T sa[3] = {h * (e0 + tE[p + 1]) + h * (e0 + tE[p - 1]), h * (e0 + tE[p + G::RS]) + h * (e0 + tE[p - G::RS]),
                     h * (e0 + tE[p + G::PS]) + h * (e0 + tE[p - G::PS])};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        T al = T(0);
        for (int ax = 0; ax < 3; ax++)
            if (ax != c) al += l * sa[ax];
        inv[((size_t)b * 3 + c) * B3 + t] = (T)g.omega / (T(1) + al);
    }
}

template <typename T>
cudaError_t launch_invdiag(const GridDev &g, const T *eta, const T *Geta, double lamdt, T *inv, cudaStream_t s) {
    if (g.nblk == 0) return cudaSuccess;
    k_invdiag<T><<<g.nblk, 512, 0, s>>>(g, eta, Geta, lamdt / (g.h * g.h), inv);
    return cudaGetLastError();
}
template cudaError_t launch_invdiag<double>(const GridDev &, const double *, const double *, double, double *, cudaStream_t);
template cudaError_t launch_invdiag<float>(const GridDev &, const float *, const float *, double, float *, cudaStream_t);

// Offset of block b's instance in a lexicographic grid of ld cells and ncomp components
// (batched hierarchies stack one such grid per instance)
__device__ __forceinline__ size_t lex_inst_offset(const GridDev &g, int b, int ncomp, int3 ld) {
    return g.inst_nblk ? (size_t)(b / g.inst_nblk) * ncomp * ((size_t)ld.x * ld.y * ld.z) : 0;
}

__device__ __forceinline__ bool inst_masked(const GridDev &g, const uint8_t *imask, int b) {
    return imask && !imask[g.inst_nblk ? b / g.inst_nblk : 0];
}

// ------------------------------------------------------------------ residual + restriction
template <typename T>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 4 : 1) k_resid_restrict(GridDev g, const T *__restrict__ e, const T *__restrict__ r,
                                                        const T *__restrict__ eta, const T *__restrict__ Ge,
                                                        const T *__restrict__ Geta, T coef, T *__restrict__ t_out,
                                                        T *__restrict__ coarse, T *__restrict__ lex, int3 ld) {
    using G = Geo<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tB = reinterpret_cast<T *>(smem_raw);
    T *tE = tB + 3 * G::CS;
    T *phi = tE + G::CS;
    T *tt = phi + G::PHI;
    __shared__ int snb[27];
    const int b = blockIdx.x;
    if (skip_block(g, b)) return;
    const int slot = g.gslot ? g.gslot[b] : -1;
    stage_nbr(snb, g.nbr, b);
    __syncthreads();
    stage_rows<T, 3, 1, G::RS, G::OFF>(tB, e, snb, slot >= 0 && Ge ? Ge + (size_t)slot * 3 * T3 : nullptr);
    stage_rows<T, 1, 1, G::RS, G::OFF>(tE, eta, snb, slot >= 0 && Geta ? Geta + (size_t)slot * T3 : nullptr);
    __syncthreads();
    all_faces_512(tB, tE, phi);
    __syncthreads();
    {
        int i, j, k;
        cell_of_thread<T>(threadIdx.x, i, j, k);
        const int cell = (k * 8 + j) * 8 + i;
        T dv[3];
        cell_div(phi, i, j, k, dv[0], dv[1], dv[2]);
        const int p = G::at(i + 1, j + 1, k + 1);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            size_t id = ((size_t)b * 3 + c) * B3 + cell;
            T v = r[id] - tB[c * G::CS + p] - coef * dv[c];
            tt[c * B3 + cell] = v;
            if (t_out) t_out[id] = v;
        }
    }
    __syncthreads();
    if ((coarse || lex) && threadIdx.x < 192) {
        const int c = threadIdx.x >> 6, q = threadIdx.x & 63;
        const int ci = q & 3, cj = (q >> 2) & 3, ck = q >> 4;
        const T *src = tt + c * B3;
        T s = 0;
        for (int dk = 0; dk < 2; dk++)
            for (int dj = 0; dj < 2; dj++)
                for (int di = 0; di < 2; di++) s += src[((2 * ck + dk) * 8 + 2 * cj + dj) * 8 + 2 * ci + di];
        s = s / T(8);
        if (coarse) {
            const int pb = g.parent[b], o = g.octant[b];
            const int x = 4 * (o & 1) + ci, y = 4 * ((o >> 1) & 1) + cj, z = 4 * (o >> 2) + ck;
            coarse[((size_t)pb * 3 + c) * B3 + (z * 8 + y) * 8 + x] = s;
        } else {
            const int x = 4 * g.origin[b * 3 + 0] + ci, y = 4 * g.origin[b * 3 + 1] + cj, z = 4 * g.origin[b * 3 + 2] + ck;
            T *lx = lex + lex_inst_offset(g, b, 3, ld);
            lx[(((size_t)c * ld.z + z) * ld.y + y) * ld.x + x] = s;
        }
    }
}

template <typename T>
cudaError_t launch_resid_restrict(const GridDev &g, const T *e, const T *r, const T *eta, const T *Ge, const T *Geta,
                                  double lamdt, T *t_out, T *coarse, T *lex, const int *ldims, cudaStream_t s) {
    if (g.nblk == 0) return cudaSuccess;
    const size_t sm = (4 * Geo<T>::CS + Geo<T>::PHI + 3 * B3) * sizeof(T);
    // set once per process (thread-safe static initialisation)
    static const bool attr = (cudaFuncSetAttribute(k_resid_restrict<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm), true);
    (void)attr;
    int3 ld = make_int3(ldims ? ldims[0] : 0, ldims ? ldims[1] : 0, ldims ? ldims[2] : 0);
    k_resid_restrict<T><<<g.nblk, 512, sm, s>>>(g, e, r, eta, Ge, Geta, (T)(lamdt / (2.0 * g.h * g.h)), t_out, coarse,
                                                lex, ld);
    return cudaGetLastError();
}
template cudaError_t launch_resid_restrict<double>(const GridDev &, const double *, const double *, const double *,
                                                   const double *, const double *, double, double *, double *, double *,
                                                   const int *, cudaStream_t);
template cudaError_t launch_resid_restrict<float>(const GridDev &, const float *, const float *, const float *,
                                                  const float *, const float *, double, float *, float *, float *,
                                                  const int *, cudaStream_t);

// ------------------------------------------------------------------ plain restriction
template <typename T>
__global__ void __launch_bounds__(512) k_restrict(GridDev g, const T *__restrict__ fine, int ncomp,
                                                  T *__restrict__ coarse, T *__restrict__ lex, int3 ld) {
    const int b = blockIdx.x;
    for (int q = threadIdx.x; q < 64 * ncomp; q += blockDim.x) {
        const int c = q >> 6, cq = q & 63;
        const int ci = cq & 3, cj = (cq >> 2) & 3, ck = cq >> 4;
        const T *src = fine + ((size_t)b * ncomp + c) * B3;
        T s = 0;
        for (int dk = 0; dk < 2; dk++)
            for (int dj = 0; dj < 2; dj++)
                for (int di = 0; di < 2; di++) s += src[((2 * ck + dk) * 8 + 2 * cj + dj) * 8 + 2 * ci + di];
        s = s / T(8);
        if (coarse) {
            const int pb = g.parent[b], o = g.octant[b];
            const int x = 4 * (o & 1) + ci, y = 4 * ((o >> 1) & 1) + cj, z = 4 * (o >> 2) + ck;
            coarse[((size_t)pb * ncomp + c) * B3 + (z * 8 + y) * 8 + x] = s;
        } else {
            const int x = 4 * g.origin[b * 3 + 0] + ci, y = 4 * g.origin[b * 3 + 1] + cj, z = 4 * g.origin[b * 3 + 2] + ck;
            T *lx = lex + lex_inst_offset(g, b, ncomp, ld);
            lx[(((size_t)c * ld.z + z) * ld.y + y) * ld.x + x] = s;
        }
    }
}

template <typename T>
cudaError_t launch_restrict(const GridDev &g, const T *fine, int ncomp, T *coarse, T *lex, const int *ldims,
                            cudaStream_t s) {
    if (g.nblk == 0) return cudaSuccess;
    int3 ld = make_int3(ldims ? ldims[0] : 0, ldims ? ldims[1] : 0, ldims ? ldims[2] : 0);
    k_restrict<T><<<g.nblk, 256, 0, s>>>(g, fine, ncomp, coarse, lex, ld);
    return cudaGetLastError();
}
template cudaError_t launch_restrict<double>(const GridDev &, const double *, int, double *, double *, const int *, cudaStream_t);
template cudaError_t launch_restrict<float>(const GridDev &, const float *, int, float *, float *, const int *, cudaStream_t);

// ------------------------------------------------------------------ prolongation
// fine += trilinear interpolation (weights 3/4, 1/4 per axis) of the coarser grid, read
// through a 6^3 window around the block's footprint in its parent (blocked) or with
// periodic wrap (lexicographic coarse grid).
template <typename T>
__global__ void __launch_bounds__(512) k_prolong_add(GridDev g, GridDev gc, const T *__restrict__ coarse,
                                                     const T *__restrict__ lex, int3 ld, T *__restrict__ fine,
                                                     int *__restrict__ err) {
    __shared__ T win[3 * 216];
    const int b = blockIdx.x;
    if (skip_block(g, b)) return;
    const int o = lex ? 0 : g.octant[b];
    const int pb = lex ? 0 : g.parent[b];
    for (int q = threadIdx.x; q < 216; q += blockDim.x) {
        const int wx = q % 6, wy = (q / 6) % 6, wz = q / 36;
        if (lex) {
            int x = 4 * g.origin[b * 3 + 0] - 1 + wx, y = 4 * g.origin[b * 3 + 1] - 1 + wy, z = 4 * g.origin[b * 3 + 2] - 1 + wz;
            x = (x + ld.x) % ld.x; y = (y + ld.y) % ld.y; z = (z + ld.z) % ld.z;
            const T *lx = lex + lex_inst_offset(g, b, 3, ld);
            for (int c = 0; c < 3; c++) win[c * 216 + q] = lx[(((size_t)c * ld.z + z) * ld.y + y) * ld.x + x];
        } else {
            int cx = 4 * (o & 1) - 1 + wx, cy = 4 * ((o >> 1) & 1) - 1 + wy, cz = 4 * (o >> 2) - 1 + wz;
            int dx = cx < 0 ? -1 : (cx > 7 ? 1 : 0), dy = cy < 0 ? -1 : (cy > 7 ? 1 : 0), dz = cz < 0 ? -1 : (cz > 7 ? 1 : 0);
            int src = gc.nbr[pb * 27 + (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
            if (src < 0) {
                if (err) *err = 1;
                for (int c = 0; c < 3; c++) win[c * 216 + q] = T(0);
            } else {
                int lx = cx - 8 * dx, ly = cy - 8 * dy, lz = cz - 8 * dz;
                for (int c = 0; c < 3; c++) win[c * 216 + q] = coarse[((size_t)src * 3 + c) * B3 + (lz * 8 + ly) * 8 + lx];
            }
        }
    }
    __syncthreads();
    const int t = threadIdx.x, i = t & 7, j = (t >> 3) & 7, k = t >> 6;
    const int wi = (i >> 1) + 1, wj = (j >> 1) + 1, wk = (k >> 1) + 1;
    const int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const T *w = win + c * 216;
        T v = 0;
        for (int ak = 0; ak < 2; ak++)
            for (int aj = 0; aj < 2; aj++)
                for (int ai = 0; ai < 2; ai++) {
                    T wt = (ai ? T(0.25) : T(0.75)) * (aj ? T(0.25) : T(0.75)) * (ak ? T(0.25) : T(0.75));
                    v += wt * w[((wk + ak * sk) * 6 + (wj + aj * sj)) * 6 + (wi + ai * si)];
                }
        fine[((size_t)b * 3 + c) * B3 + t] += v;
    }
}

template <typename T>
cudaError_t launch_prolong_add(const GridDev &g, const GridDev *gc, const T *coarse, const T *lex, const int *ldims,
                               T *fine, int *err, cudaStream_t s) {
    if (g.nblk == 0) return cudaSuccess;
    int3 ld = make_int3(ldims ? ldims[0] : 0, ldims ? ldims[1] : 0, ldims ? ldims[2] : 0);
    GridDev c = gc ? *gc : GridDev();
    k_prolong_add<T><<<g.nblk, 512, 0, s>>>(g, c, coarse, lex, ld, fine, err);
    return cudaGetLastError();
}
template cudaError_t launch_prolong_add<double>(const GridDev &, const GridDev *, const double *, const double *,
                                                const int *, double *, int *, cudaStream_t);
template cudaError_t launch_prolong_add<float>(const GridDev &, const GridDev *, const float *, const float *,
                                               const int *, float *, int *, cudaStream_t);

// Prolongation for a coarse grid whose blocks' 8 children are the fine blocks 8c .. 8c+7 in
// octant order (Morton-ordered complete grids): one thread block per coarse block stages the
// coarse block and its 1-cell halo once (10^3, as the stencil kernels do) and adds the
// trilinear interpolant (3/4, 1/4 per axis, the weights of k_prolong_add) to all 4096 cells of
// the 8 children, one child block per pass of its 512 threads.
template <typename T>
__global__ void __launch_bounds__(512) k_prolong_add8(GridDev gc, const T *__restrict__ coarse, T *__restrict__ fine) {
    using G = Geo<T>;
    __shared__ __align__(16) T tC[3 * G::CS];
    __shared__ int snb[27];
    const int c = blockIdx.x;
    if (skip_block(gc, c)) return;
    stage_nbr(snb, gc.nbr, c);
    __syncthreads();
    stage_rows<T, 3, 1, G::RS, G::OFF>(tC, coarse, snb, nullptr);
    __syncthreads();
    const int t = threadIdx.x, lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
    for (int o = 0; o < 8; o++) {
        const int fx = lx + 8 * (o & 1), fy = ly + 8 * ((o >> 1) & 1), fz = lz + 8 * (o >> 2);
        const int cx = fx >> 1, cy = fy >> 1, cz = fz >> 1;
        const int sx = (fx & 1) ? 1 : -1, sy = (fy & 1) ? 1 : -1, sz = (fz & 1) ? 1 : -1;
        const int p = G::at(cx + 1, cy + 1, cz + 1);
        const size_t fb = ((size_t)(8 * c + o) * 3) * B3 + t;
#pragma unroll
        for (int comp = 0; comp < 3; comp++) {
            const T *w = tC + comp * G::CS;
            T v = 0;
            for (int ak = 0; ak < 2; ak++)
                for (int aj = 0; aj < 2; aj++)
                    for (int ai = 0; ai < 2; ai++) {
                        const T wt = (ai ? T(0.25) : T(0.75)) * (aj ? T(0.25) : T(0.75)) * (ak ? T(0.25) : T(0.75));
                        v += wt * w[p + ak * sz * G::PS + aj * sy * G::RS + ai * sx];
                    }
            fine[fb + (size_t)comp * B3] += v;
        }
    }
}

template <typename T>
cudaError_t launch_prolong_add8(const GridDev &gc, const T *coarse, T *fine, cudaStream_t s) {
    if (gc.nblk == 0) return cudaSuccess;
    k_prolong_add8<T><<<gc.nblk, 512, 0, s>>>(gc, coarse, fine);
    return cudaGetLastError();
}
template cudaError_t launch_prolong_add8<double>(const GridDev &, const double *, double *, cudaStream_t);
template cudaError_t launch_prolong_add8<float>(const GridDev &, const float *, float *, cudaStream_t);

// ------------------------------------------------------------------ coarse-fine ghosts
// Ghost slot of a level-l block: every halo cell gets the tri-quadratic interpolant of the
// parent's 3x3x3 coarse neighbourhood at the child's centre (offset s h_c/4 per axis):
//   f0 + sum_d [s_d (f+ - f-)/8 + (f+ - 2 f0 + f-)/32] + sum_{d<e} s_d s_e (cross diff)/64.
// The coarse window is [4o-2, 4o+6) per axis in parent-local cells.
template <typename TS_, typename TD>
__global__ void __launch_bounds__(512) k_ghost_fill(GridDev g, GridDev gc, const TS_ *__restrict__ coarse, int ncomp,
                                                    TD *__restrict__ ghost, int *__restrict__ err) {
    __shared__ double win[3 * 512];
    const int sl = blockIdx.x;
    const int b = g.slot_block[sl];
    if (skip_block(g, b)) return;
    const int pb = g.parent[b], o = g.octant[b];
    const int ox = 4 * (o & 1), oy = 4 * ((o >> 1) & 1), oz = 4 * (o >> 2);
    for (int q = threadIdx.x; q < 512; q += blockDim.x) {
        const int wx = q & 7, wy = (q >> 3) & 7, wz = q >> 6;
        int cx = ox - 2 + wx, cy = oy - 2 + wy, cz = oz - 2 + wz;
        int dx = cx < 0 ? -1 : (cx > 7 ? 1 : 0), dy = cy < 0 ? -1 : (cy > 7 ? 1 : 0), dz = cz < 0 ? -1 : (cz > 7 ? 1 : 0);
        int src = gc.nbr[pb * 27 + (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
        if (src < 0) {
            if (err) *err = 1;
            for (int c = 0; c < ncomp; c++) win[c * 512 + q] = 0.0;
        } else {
            int lx = cx - 8 * dx, ly = cy - 8 * dy, lz = cz - 8 * dz;
            for (int c = 0; c < ncomp; c++)
                win[c * 512 + q] = (double)coarse[((size_t)src * ncomp + c) * B3 + (lz * 8 + ly) * 8 + lx];
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < T3; idx += blockDim.x) {
        const int ti = idx % TS, tj = (idx / TS) % TS, tk = idx / (TS * TS);
        const int gi = ti - 1, gj = tj - 1, gk = tk - 1;
        const int outx = gi < 0 || gi > 7, outy = gj < 0 || gj > 7, outz = gk < 0 || gk > 7;
        const int nout = outx + outy + outz;
        if (nout == 0 || nout == 3) continue;
        const int w[3] = {(gi >> 1) + 2, (gj >> 1) + 2, (gk >> 1) + 2};
        const double sg[3] = {(gi & 1) ? 1.0 : -1.0, (gj & 1) ? 1.0 : -1.0, (gk & 1) ? 1.0 : -1.0};
        const int st[3] = {1, 8, 64};
        const int w0 = (w[2] * 8 + w[1]) * 8 + w[0];
        for (int c = 0; c < ncomp; c++) {
            const double *W = win + c * 512;
            const double f0 = W[w0];
            double val = f0;
            for (int d = 0; d < 3; d++) {
                double fp = W[w0 + st[d]], fm = W[w0 - st[d]];
                val += sg[d] * (fp - fm) / 8.0 + (fp - 2.0 * f0 + fm) / 32.0;
            }
            for (int d = 0; d < 3; d++)
                for (int e = d + 1; e < 3; e++) {
                    double x4 = (W[w0 + st[d] + st[e]] - W[w0 + st[d] - st[e]]) - (W[w0 - st[d] + st[e]] - W[w0 - st[d] - st[e]]);
                    val += sg[d] * sg[e] * x4 / 64.0;
                }
            ghost[((size_t)sl * ncomp + c) * T3 + idx] = (TD)val;
        }
    }
}

template <typename TS_, typename TD>
cudaError_t launch_ghost_fill(const GridDev &g, const GridDev &gc, const TS_ *coarse, int ncomp, TD *ghost, int *err,
                              cudaStream_t s) {
    if (g.nslot == 0) return cudaSuccess;
    k_ghost_fill<TS_, TD><<<g.nslot, 512, 0, s>>>(g, gc, coarse, ncomp, ghost + (size_t)g.slot0 * ncomp * T3, err);
    return cudaGetLastError();
}
template cudaError_t launch_ghost_fill<double, double>(const GridDev &, const GridDev &, const double *, int, double *,
                                                       int *, cudaStream_t);
template cudaError_t launch_ghost_fill<double, float>(const GridDev &, const GridDev &, const double *, int, float *,
                                                      int *, cudaStream_t);
template cudaError_t launch_ghost_fill<float, float>(const GridDev &, const GridDev &, const float *, int, float *,
                                                     int *, cudaStream_t);

// ------------------------------------------------------------------ sync down, update
template <typename T>
__global__ void __launch_bounds__(512) k_sync_down(GridDev gc, T *__restrict__ Bc, const T *__restrict__ Bf) {
    const int b = blockIdx.x;
    if (!gc.covered[b] || skip_block(gc, b)) return;
    const int t = threadIdx.x, i = t & 7, j = (t >> 3) & 7, k = t >> 6;
    const int oc = (i >> 2) | ((j >> 2) << 1) | ((k >> 2) << 2);
    const int ch = gc.child[b * 8 + oc];
    const int fi = 2 * (i & 3), fj = 2 * (j & 3), fk = 2 * (k & 3);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const T *src = Bf + ((size_t)ch * 3 + c) * B3;
        T s = 0;
        for (int dk = 0; dk < 2; dk++)
            for (int dj = 0; dj < 2; dj++)
                for (int di = 0; di < 2; di++) s += src[((fk + dk) * 8 + fj + dj) * 8 + fi + di];
        Bc[((size_t)b * 3 + c) * B3 + t] = s / T(8);
    }
}

template <typename T>
cudaError_t launch_sync_down(const GridDev &gc, T *Bc, const T *Bf, cudaStream_t s) {
    if (gc.nblk == 0) return cudaSuccess;
    k_sync_down<T><<<gc.nblk, 512, 0, s>>>(gc, Bc, Bf);
    return cudaGetLastError();
}
template cudaError_t launch_sync_down<double>(const GridDev &, double *, const double *, cudaStream_t);
template cudaError_t launch_sync_down<float>(const GridDev &, float *, const float *, cudaStream_t);

// x += y on leaf blocks (inner correction accumulation)
template <typename T>
__global__ void __launch_bounds__(512) k_axpy_leaf(GridDev g, T *__restrict__ x, const T *__restrict__ y,
                                                   const uint8_t *__restrict__ imask) {
    const int b = blockIdx.x;
    if ((g.covered && g.covered[b]) || inst_masked(g, imask, b)) return;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        size_t id = ((size_t)b * 3 + c) * B3 + threadIdx.x;
        x[id] += y[id];
    }
}

template <typename T>
cudaError_t launch_axpy_leaf(const GridDev &g, T *x, const T *y, const uint8_t *imask, cudaStream_t s) {
    if (g.nblk == 0) return cudaSuccess;
    k_axpy_leaf<T><<<g.nblk, 512, 0, s>>>(g, x, y, imask);
    return cudaGetLastError();
}
template cudaError_t launch_axpy_leaf<float>(const GridDev &, float *, const float *, const uint8_t *, cudaStream_t);
template cudaError_t launch_axpy_leaf<double>(const GridDev &, double *, const double *, const uint8_t *, cudaStream_t);

template <typename T>
__global__ void __launch_bounds__(512) k_update(GridDev g, double *__restrict__ B, const T *__restrict__ e,
                                                const uint8_t *__restrict__ imask) {
    const int b = blockIdx.x;
    if ((g.covered && g.covered[b]) || inst_masked(g, imask, b)) return;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        size_t id = ((size_t)b * 3 + c) * B3 + threadIdx.x;
        B[id] += (double)e[id];
    }
}

template <typename T>
cudaError_t launch_update(const GridDev &g, double *B, const T *e, const uint8_t *imask, cudaStream_t s) {
    if (g.nblk == 0) return cudaSuccess;
    k_update<T><<<g.nblk, 512, 0, s>>>(g, B, e, imask);
    return cudaGetLastError();
}
template cudaError_t launch_update<double>(const GridDev &, double *, const double *, const uint8_t *, cudaStream_t);
template cudaError_t launch_update<float>(const GridDev &, double *, const float *, const uint8_t *, cudaStream_t);

__global__ void __launch_bounds__(512) k_zero_covered(GridDev g, double *__restrict__ x) {
    const int b = blockIdx.x;
    if (!(g.covered && g.covered[b])) return;
    for (int c = 0; c < 3; c++) x[((size_t)b * 3 + c) * B3 + threadIdx.x] = 0.0;
}

cudaError_t launch_zero_covered(const GridDev &g, double *x, cudaStream_t s) {
    if (g.nblk == 0 || !g.covered) return cudaSuccess;
    k_zero_covered<<<g.nblk, 512, 0, s>>>(g, x);
    return cudaGetLastError();
}

// Deterministic reduction of per-block partials {sum R^2 dV, sum S^2 dV, max |R|}: every
// thread block folds a fixed contiguous chunk in a fixed order, and the last block to finish
// (atomic ticket) folds the per-chunk results in chunk order.
constexpr int NRED = 128;
__global__ void __launch_bounds__(256) k_norm_reduce(const double *__restrict__ part, int n, double *__restrict__ chunk,
                                                     unsigned int *__restrict__ ticket, double *__restrict__ out,
                                                     double *__restrict__ host_out, const int *__restrict__ err) {
    __shared__ double red[32];
    __shared__ bool last;
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * per, hi = min(n, lo + per);
    double a = 0.0, b = 0.0, m = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        a += part[i * 3 + 0];
        b += part[i * 3 + 1];
        m = fmax(m, part[i * 3 + 2]);
    }
    double sa = block_sum(a, red);
    double sb = block_sum(b, red);
    double sm = block_max(m, red);
    if (threadIdx.x == 0) {
        chunk[blockIdx.x * 3 + 0] = sa;
        chunk[blockIdx.x * 3 + 1] = sb;
        chunk[blockIdx.x * 3 + 2] = sm;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    a = b = m = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        a += __ldcg(chunk + i * 3 + 0);
        b += __ldcg(chunk + i * 3 + 1);
        m = fmax(m, __ldcg(chunk + i * 3 + 2));
    }
    sa = block_sum(a, red);
    sb = block_sum(b, red);
    sm = block_max(m, red);
    if (threadIdx.x == 0) {
        out[0] = sa;
        out[1] = sb;
        out[2] = sm;
        if (host_out) {  // pinned host memory mapped into the device: no copy needed to read them
            host_out[0] = sa;
            host_out[1] = sb;
            host_out[2] = sm;
            reinterpret_cast<volatile int *>(host_out + 4)[0] = err ? *err : 0;
        }
        *ticket = 0u;
    }
}

// scratch: NRED * 3 doubles followed by one unsigned ticket (zero on first use)
cudaError_t launch_norm_reduce(const double *partials, int nblocks, double *scratch, double *out, cudaStream_t s,
                               double *host_out, const int *err) {
    int grid = nblocks < NRED * 64 ? (nblocks + 63) / 64 : NRED;
    k_norm_reduce<<<grid, 256, 0, s>>>(partials, nblocks, scratch, (unsigned int *)(scratch + 3 * NRED), out, host_out, err);
    return cudaGetLastError();
}

// One thread block per instance; its level ranges are folded in level order, each range in a
// fixed thread-strided order, so the result does not depend on the other instances.
__global__ void __launch_bounds__(256) k_norm_inst(const double *__restrict__ part, InstRanges R,
                                                   double *__restrict__ out) {
    __shared__ double red[32];
    const int q = blockIdx.x;
    double a = 0.0, b = 0.0, m = 0.0;
    for (int l = 0; l < R.nlev; l++) {
        const int lo = R.off[l] + q * R.n[l], hi = lo + R.n[l];
        for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            a += part[i * 3 + 0];
            b += part[i * 3 + 1];
            m = fmax(m, part[i * 3 + 2]);
        }
    }
    const double sa = block_sum(a, red);
    const double sb = block_sum(b, red);
    const double sm = block_max(m, red);
    if (threadIdx.x == 0) {
        out[q * 4 + 0] = sa;
        out[q * 4 + 1] = sb;
        out[q * 4 + 2] = sm;
        out[q * 4 + 3] = 0.0;
    }
}

cudaError_t launch_norm_inst(const double *partials, const InstRanges &R, int ninst, double *out, cudaStream_t s) {
    if (ninst <= 0) return cudaSuccess;
    k_norm_inst<<<ninst, 256, 0, s>>>(partials, R, out);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(512) k_scale_blocks(const double *__restrict__ src, double *__restrict__ dst,
                                                      const double *__restrict__ scale) {
    const size_t id = (size_t)blockIdx.x * B3 + threadIdx.x;
    dst[id] = src[id] * scale[blockIdx.x];
}

cudaError_t launch_scale_blocks(const double *src, double *dst, const double *scale, int nblk, cudaStream_t s) {
    if (nblk <= 0) return cudaSuccess;
    k_scale_blocks<<<nblk, 512, 0, s>>>(src, dst, scale);
    return cudaGetLastError();
}

template <typename TS_, typename TD>
__global__ void k_convert(const TS_ *__restrict__ src, TD *__restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (TD)src[i];
}

template <typename TS_, typename TD>
cudaError_t launch_convert(const TS_ *src, TD *dst, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int grid = (int)((n + 255) / 256);
    if (grid > 152 * 32) grid = 152 * 32;
    k_convert<TS_, TD><<<grid, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(const double *, float *, size_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double *, double *, size_t, cudaStream_t);

// ------------------------------------------------------------------ Krylov vector kernels
// Vectors are block fields [nblk][3][512]; inner products are volume weighted over leaf
// blocks (weight w_b = h^3, 0 for covered blocks), the norm of the convergence tests.
// The number of vectors NV is a template parameter (one instantiation per count, chosen at
// launch), so a thread holds exactly NV + 1 partial sums: with a run-time count the compiler
// kept the 13 sums of the largest case, which cost occupancy (76 registers).
// One warp per 8^3 block: each lane forms 12 float4 products per column in float32, the warp
// reduces them by shuffles and lane 0 weights the sum in float64.
template <int NV>
__device__ __forceinline__ void warp_block_dots(const float *__restrict__ w, const VecSet &V, int b, int lane,
                                                double wt, double out[NV + 1]) {
    float f[NV + 1];
#pragma unroll
    for (int i = 0; i <= NV; i++) f[i] = 0.f;
    if (wt != 0.0) {
        const float4 *w4 = reinterpret_cast<const float4 *>(w + (size_t)b * 1536);
#pragma unroll 1
        for (int s = 0; s < 12; s++) {
            const float4 x = w4[lane + 32 * s];
            f[NV] += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
#pragma unroll
            for (int i = 0; i < NV; i++) {
                const float4 v = reinterpret_cast<const float4 *>(V.v[i] + (size_t)b * 1536)[lane + 32 * s];
                f[i] += x.x * v.x + x.y * v.y + x.z * v.z + x.w * v.w;
            }
        }
    }
#pragma unroll
    for (int i = 0; i <= NV; i++) {
        float v = f[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        out[i] = (double)v * wt;
    }
}

// the 8 warps of a thread block are folded in warp order into part[blockIdx][col]
template <int NV>
__global__ void __launch_bounds__(256) k_mdot(const float *__restrict__ w, VecSet V, const double *__restrict__ wb,
                                              int nblk, double *__restrict__ part, const int *__restrict__ gate) {
    if (gate && !*gate) return;
    __shared__ double sred[8][NV + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * 8 + warp;
    double d[NV + 1];
    warp_block_dots<NV>(w, V, b < nblk ? b : 0, lane, b < nblk ? wb[b] : 0.0, d);
    if (lane == 0)
        for (int i = 0; i <= NV; i++) sred[warp][i] = d[i];
    __syncthreads();
    if (threadIdx.x <= NV) {
        double a = 0.0;
        for (int q = 0; q < 8; q++) a += sred[q][threadIdx.x];
        part[(size_t)blockIdx.x * (NV + 1) + threadIdx.x] = a;
    }
}

// column sums of part[nrow][ncol] in a fixed order (one thread block per column)
__global__ void __launch_bounds__(256) k_colsum(const double *__restrict__ part, int nrow, int ncol, double *__restrict__ out,
                                                const int *__restrict__ gate, double *__restrict__ host_out) {
    if (gate && !*gate) return;
    __shared__ double red[32];
    const int c = blockIdx.x;
    double a = 0.0;
    for (int b = threadIdx.x; b < nrow; b += blockDim.x) a += part[(size_t)b * ncol + c];
    double s = block_sum(a, red);
    if (threadIdx.x == 0) {
        out[c] = s;
        if (host_out) host_out[c] = s;  // mapped pinned host memory
    }
}

// dst = (src - sum_i c_i v_i) * scale (dst may equal src; src null reads as 0); float4 over n/4 groups
template <int NV>
__global__ void __launch_bounds__(256) k_maxpy(float4 *dst, const float4 *src, VecSet V, float scale, size_t n4) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n4; q += (size_t)gridDim.x * blockDim.x) {
        float4 x = src ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < NV; i++) {
            const float4 v = reinterpret_cast<const float4 *>(V.v[i])[q];
            const float c = V.c[i];
            x.x -= c * v.x;
            x.y -= c * v.y;
            x.z -= c * v.z;
            x.w -= c * v.w;
        }
        x.x *= scale;
        x.y *= scale;
        x.z *= scale;
        x.w *= scale;
        dst[q] = x;
    }
}

// one instantiation per vector count 0 .. KMAX
#define OHM_NV_SWITCH(k, CALL)   \
    switch (k) {                 \
        case 0: CALL(0); break;  \
        case 1: CALL(1); break;  \
        case 2: CALL(2); break;  \
        case 3: CALL(3); break;  \
        case 4: CALL(4); break;  \
        case 5: CALL(5); break;  \
        case 6: CALL(6); break;  \
        case 7: CALL(7); break;  \
        case 8: CALL(8); break;  \
        case 9: CALL(9); break;  \
        case 10: CALL(10); break; \
        case 11: CALL(11); break; \
        default: CALL(12); break; \
    }

cudaError_t launch_mdot(const float *w, const VecSet &V, const double *wb, int nblk, double *part, double *out,
                        cudaStream_t s, const int *gate, double *host_out) {
    const int grid = (nblk + 7) / 8;
#define OHM_MDOT(N) k_mdot<N><<<grid, 256, 0, s>>>(w, V, wb, nblk, part, gate)
    OHM_NV_SWITCH(V.k, OHM_MDOT)
#undef OHM_MDOT
    k_colsum<<<V.k + 1, 256, 0, s>>>(part, grid, V.k + 1, out, gate, host_out);
    return cudaGetLastError();
}

// float64 Krylov vectors: one warp per block for the products (double2 loads, float64 sums), a
// grid-stride loop for the updates
template <int NV>
__global__ void __launch_bounds__(256) k_mdot_d(const double *__restrict__ w, VecSetD V, const double *__restrict__ wb,
                                                int nblk, double *__restrict__ part) {
    __shared__ double sred[8][NV + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * 8 + warp;
    double f[NV + 1];
#pragma unroll
    for (int i = 0; i <= NV; i++) f[i] = 0.0;
    const double wt = b < nblk ? wb[b] : 0.0;
    if (wt != 0.0) {
        const double2 *w2 = reinterpret_cast<const double2 *>(w + (size_t)b * 1536);
#pragma unroll 1
        for (int q = lane; q < 768; q += 32) {
            const double2 x = w2[q];
            f[NV] = fma(x.x, x.x, fma(x.y, x.y, f[NV]));
#pragma unroll
            for (int i = 0; i < NV; i++) {
                const double2 v = reinterpret_cast<const double2 *>(V.v[i] + (size_t)b * 1536)[q];
                f[i] = fma(x.x, v.x, fma(x.y, v.y, f[i]));
            }
        }
    }
#pragma unroll
    for (int i = 0; i <= NV; i++) {
        double v = f[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sred[warp][i] = v * wt;
    }
    __syncthreads();
    if (threadIdx.x <= NV) {
        double a = 0.0;
        for (int q = 0; q < 8; q++) a += sred[q][threadIdx.x];
        part[(size_t)blockIdx.x * (NV + 1) + threadIdx.x] = a;
    }
}

template <int NV>
__global__ void __launch_bounds__(256) k_maxpy_d(double2 *dst, const double2 *src, VecSetD V, double scale, size_t n2) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n2; q += (size_t)gridDim.x * blockDim.x) {
        double2 x = src ? src[q] : make_double2(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < NV; i++) {
            const double2 v = reinterpret_cast<const double2 *>(V.v[i])[q];
            x.x = fma(-V.c[i], v.x, x.x);
            x.y = fma(-V.c[i], v.y, x.y);
        }
        x.x *= scale;
        x.y *= scale;
        dst[q] = x;
    }
}

cudaError_t launch_mdot(const double *w, const VecSetD &V, const double *wb, int nblk, double *part, double *out,
                        cudaStream_t s, double *host_out) {
    const int grid = (nblk + 7) / 8;
#define OHM_MDOTD(N) k_mdot_d<N><<<grid, 256, 0, s>>>(w, V, wb, nblk, part)
    OHM_NV_SWITCH(V.k, OHM_MDOTD)
#undef OHM_MDOTD
    k_colsum<<<V.k + 1, 256, 0, s>>>(part, grid, V.k + 1, out, nullptr, host_out);
    return cudaGetLastError();
}

cudaError_t launch_maxpy(double *dst, const double *src, const VecSetD &V, double scale, size_t n, cudaStream_t s) {
    const size_t n2 = n / 2;
    const int grid = (int)std::min<size_t>((n2 + 255) / 256, 152 * 16);
    double2 *d2 = reinterpret_cast<double2 *>(dst);
    const double2 *s2 = reinterpret_cast<const double2 *>(src);
#define OHM_MAXPYD(N) k_maxpy_d<N><<<grid, 256, 0, s>>>(d2, s2, V, scale, n2)
    OHM_NV_SWITCH(V.k, OHM_MAXPYD)
#undef OHM_MAXPYD
    return cudaGetLastError();
}

// column sums of part[ncol][nrow] (column-major) in a fixed order, one thread block per column
__global__ void __launch_bounds__(1024) k_colsum_cm(const double *__restrict__ part, int nrow, double *__restrict__ out,
                                                    double *__restrict__ host_out) {
    __shared__ double red[32];
    const double *col = part + (size_t)blockIdx.x * nrow;
    double a = 0.0;
    for (int b = threadIdx.x; b < nrow; b += blockDim.x) a += col[b];
    const double s = block_sum(a, red);
    if (threadIdx.x == 0) {
        out[blockIdx.x] = s;
        if (host_out) host_out[blockIdx.x] = s;  // mapped pinned host memory
    }
}

// w = L z on block pairs (the float32 operator of the inner solve) together with <w, v_i> and
// <w, w> of the FGMRES Arnoldi step: one pass instead of the operator and the multi-dot
cudaError_t launch_pair_apply_dots(const GridDev &g, const float *X, const float *eta, double kc, float *w,
                                   const VecSet &V, double wt, double *part, double *out, double *host_out,
                                   cudaStream_t s) {
    if (g.nblk == 0) return cudaSuccess;
    const size_t sm = 4 * G18::CS * sizeof(float);
    const int npair = g.nblk / 2;
#define OHM_PAIRDOT(N)                                                                                          \
    {                                                                                                          \
        static const bool attr_ =                                                                              \
            (cudaFuncSetAttribute(k_pair_op<true, false, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm), \
             true);                                                                                            \
        (void)attr_;                                                                                           \
        k_pair_op<true, false, N><<<npair, 512, sm, s>>>(g, X, nullptr, eta, (float)kc, w, nullptr, V, wt, part);  \
    }
    OHM_NV_SWITCH(V.k, OHM_PAIRDOT)
#undef OHM_PAIRDOT
    k_colsum_cm<<<V.k + 1, 1024, 0, s>>>(part, npair, out, host_out);
    return cudaGetLastError();
}

cudaError_t launch_maxpy(float *dst, const float *src, const VecSet &V, float scale, size_t n, cudaStream_t s) {
    const size_t n4 = n / 4;  // fields are whole 8^3 blocks: n is a multiple of 1536
    const int grid = (int)std::min<size_t>((n4 + 255) / 256, 152 * 16);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#define OHM_MAXPY(N) k_maxpy<N><<<grid, 256, 0, s>>>(d4, s4, V, scale, n4)
    OHM_NV_SWITCH(V.k, OHM_MAXPY)
#undef OHM_MAXPY
    return cudaGetLastError();
}


// Per-instance Krylov vector kernels of batched hierarchies.  Block partials: one warp per
// block writes its weighted products (no folding across blocks, so no sum mixes instances).
template <int NV>
__global__ void __launch_bounds__(256) k_mdot_blocks(const float *__restrict__ w, VecSet V, const double *__restrict__ wb,
                                                     int nblk, double *__restrict__ part, const int *__restrict__ gate) {
    if (gate && !*gate) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * 8 + warp;
    if (b >= nblk) return;
    double d[NV + 1];
    warp_block_dots<NV>(w, V, b, lane, wb[b], d);
    if (lane == 0)
        for (int i = 0; i <= NV; i++) part[(size_t)b * (NV + 1) + i] = d[i];
}

// out[q][c] = sum of part[b][c] over instance q's blocks of every level, in a fixed order
__global__ void __launch_bounds__(256) k_colsum_inst(const double *__restrict__ part, InstRanges R, int ncol,
                                                     double *__restrict__ out, const int *__restrict__ gate) {
    if (gate && !*gate) return;
    __shared__ double red[32];
    const int q = blockIdx.x;
    for (int c = 0; c < ncol; c++) {
        double a = 0.0;
        for (int l = 0; l < R.nlev; l++) {
            const int lo = R.off[l] + q * R.n[l], hi = lo + R.n[l];
            for (int b = lo + threadIdx.x; b < hi; b += blockDim.x) a += part[(size_t)b * ncol + c];
        }
        const double sum = block_sum(a, red);
        if (threadIdx.x == 0) out[(size_t)q * (KMAX + 1) + c] = sum;
    }
}

cudaError_t launch_mdot_inst(const float *w, const VecSet &V, const double *wb, int nblk, const InstRanges &R, int ninst,
                             double *part, double *out, cudaStream_t s, const int *gate) {
#define OHM_MDOTB(N) k_mdot_blocks<N><<<(nblk + 7) / 8, 256, 0, s>>>(w, V, wb, nblk, part, gate)
    OHM_NV_SWITCH(V.k, OHM_MDOTB)
#undef OHM_MDOTB
    k_colsum_inst<<<ninst, 256, 0, s>>>(part, R, V.k + 1, out, gate);
    return cudaGetLastError();
}

// dst = (src - sum_i c[q][i] v_i) * c[q][KMAX] with q the instance of the element's block;
// terms whose coefficient is 0 are skipped (their vectors may hold anything for that instance)
template <int NV>
__global__ void __launch_bounds__(256) k_maxpy_inst(float4 *dst, const float4 *src, VecSet V,
                                                    const float *__restrict__ coef, const int *__restrict__ binst,
                                                    size_t n4, const int *__restrict__ gate) {
    if (gate && !*gate) return;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n4; e += (size_t)gridDim.x * blockDim.x) {
        const float *cq = coef + (size_t)binst[e / 384] * (KMAX + 1);
        float4 x = src[e];
#pragma unroll
        for (int i = 0; i < NV; i++) {
            const float c = cq[i];
            if (c != 0.f) {
                const float4 v = reinterpret_cast<const float4 *>(V.v[i])[e];
                x.x -= c * v.x;
                x.y -= c * v.y;
                x.z -= c * v.z;
                x.w -= c * v.w;
            }
        }
        const float sc = cq[KMAX];
        x.x *= sc;
        x.y *= sc;
        x.z *= sc;
        x.w *= sc;
        dst[e] = x;
    }
}

cudaError_t launch_maxpy_inst(float *dst, const float *src, const VecSet &V, const float *coef, const int *binst,
                              size_t n, cudaStream_t s, const int *gate) {
    const size_t n4 = n / 4;
    const int grid = (int)std::min<size_t>((n4 + 255) / 256, 152 * 16);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#define OHM_MAXPYI(N) k_maxpy_inst<N><<<grid, 256, 0, s>>>(d4, s4, V, coef, binst, n4, gate)
    OHM_NV_SWITCH(V.k, OHM_MAXPYI)
#undef OHM_MAXPYI
    return cudaGetLastError();
}

// ------------------------------------------------------------------ coarsest grids
// Lexicographic periodic grids below the last blocked grid, all handled by one thread block per
// instance with a barrier between phases.  Face flux and divergence as above, with periodic wrap.
template <typename T>
struct LexGrid {
    int nx, ny, nz;
    __device__ __forceinline__ int wrap(int v, int n) const { return v < 0 ? v + n : (v >= n ? v - n : v); }
    __device__ __forceinline__ size_t id(int c, int x, int y, int z) const {
        return (((size_t)c * nz + wrap(z, nz)) * ny + wrap(y, ny)) * nx + wrap(x, nx);
    }
};

template <typename T>
__device__ __forceinline__ void lex_face(const LexGrid<T> &G, const T *B, const T *E, int x, int y, int z, int a,
                                         T &phi1, T &phi2) {
    int o[3] = {0, 0, 0};
    o[a] = 1;
    const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;
    T es = E[G.id(0, x, y, z)] + E[G.id(0, x + o[0], y + o[1], z + o[2])];
    T ph[2];
    const int bb[2] = {b1, b2};
    for (int q = 0; q < 2; q++) {
        int b = bb[q];
        int e[3] = {0, 0, 0};
        e[b] = 1;
        T n = B[G.id(b, x + o[0], y + o[1], z + o[2])] - B[G.id(b, x, y, z)];
        T tr = (B[G.id(a, x + o[0] + e[0], y + o[1] + e[1], z + o[2] + e[2])] + B[G.id(a, x + e[0], y + e[1], z + e[2])]) -
               (B[G.id(a, x + o[0] - e[0], y + o[1] - e[1], z + o[2] - e[2])] + B[G.id(a, x - e[0], y - e[1], z - e[2])]);
        ph[q] = es * (T(0.25) * tr - n);
    }
    phi1 = ph[0];
    phi2 = ph[1];
}

template <typename T>
__device__ __forceinline__ void lex_div(const LexGrid<T> &G, const T *B, const T *E, int x, int y, int z, T dv[3]) {
    T xl1, xl2, xh1, xh2, yl1, yl2, yh1, yh2, zl1, zl2, zh1, zh2;
    lex_face(G, B, E, x - 1, y, z, 0, xl1, xl2);
    lex_face(G, B, E, x, y, z, 0, xh1, xh2);
    lex_face(G, B, E, x, y - 1, z, 1, yl1, yl2);
    lex_face(G, B, E, x, y, z, 1, yh1, yh2);
    lex_face(G, B, E, x, y, z - 1, 2, zl1, zl2);
    lex_face(G, B, E, x, y, z, 2, zh1, zh2);
    dv[0] = (yh1 - yl1) + (zh1 - zl1);
    dv[1] = (xh1 - xl1) + (zh2 - zl2);
    dv[2] = (xh2 - xl2) + (yh2 - yl2);
}

template <typename T>
__device__ void lex_sweeps(const SmallDev<T> &sm, int s, double lamdt, int nsweep) {
    LexGrid<T> G{sm.dims[s][0], sm.dims[s][1], sm.dims[s][2]};
    const int n = G.nx * G.ny * G.nz;
    const T coef = (T)(lamdt / (2.0 * sm.h[s] * sm.h[s]));
    T *e = sm.e[s], *d = sm.t[s];
    const T *r = sm.r[s], *E = sm.eta[s], *inv = sm.inv[s];
    for (int sw = 0; sw < nsweep; sw++)
        for (int colour = 0; colour < 2; colour++) {
            for (int q = threadIdx.x; q < n; q += blockDim.x) {
                int x = q % G.nx, y = (q / G.nx) % G.ny, z = q / (G.nx * G.ny);
                if (((x + y + z) & 1) != colour) continue;
                T dv[3];
                lex_div(G, e, E, x, y, z, dv);
                for (int c = 0; c < 3; c++) {
                    size_t id = (size_t)c * n + q;
                    d[id] = (r[id] - e[id] - coef * dv[c]) * inv[id];
                }
            }
            __syncthreads();
            for (int q = threadIdx.x; q < n; q += blockDim.x) {
                int x = q % G.nx, y = (q / G.nx) % G.ny, z = q / (G.nx * G.ny);
                if (((x + y + z) & 1) != colour) continue;
                for (int c = 0; c < 3; c++) e[(size_t)c * n + q] += d[(size_t)c * n + q];
            }
            __syncthreads();
        }
}

// the grids of instance blockIdx.x
template <typename T>
__device__ __forceinline__ SmallDev<T> small_instance(const SmallDev<T> &in) {
    SmallDev<T> sm = in;
    const size_t q = blockIdx.x;
    for (int s = 0; s < sm.n; s++) {
        const size_t cells = (size_t)sm.dims[s][0] * sm.dims[s][1] * sm.dims[s][2];
        sm.e[s] += q * 3 * cells;
        sm.r[s] += q * 3 * cells;
        sm.t[s] += q * 3 * cells;
        sm.inv[s] += q * 3 * cells;
        sm.eta[s] += q * cells;
    }
    return sm;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_bottom(SmallDev<T> sm_all, double lamdt, int nu1, int nu2, int nc) {
    if (sm_all.imask && !sm_all.imask[blockIdx.x]) return;
    const SmallDev<T> sm = small_instance(sm_all);
    // e on the first small grid starts from zero
    {
        const int n0 = sm.dims[0][0] * sm.dims[0][1] * sm.dims[0][2];
        for (int q = threadIdx.x; q < 3 * n0; q += blockDim.x) sm.e[0][q] = T(0);
        __syncthreads();
    }
    int s = 0;
    for (; s < sm.n - 1; s++) {
        lex_sweeps(sm, s, lamdt, nu1);
        LexGrid<T> G{sm.dims[s][0], sm.dims[s][1], sm.dims[s][2]};
        LexGrid<T> C{sm.dims[s + 1][0], sm.dims[s + 1][1], sm.dims[s + 1][2]};
        const int n = G.nx * G.ny * G.nz, nc_ = C.nx * C.ny * C.nz;
        const T coef = (T)(lamdt / (2.0 * sm.h[s] * sm.h[s]));
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            int x = q % G.nx, y = (q / G.nx) % G.ny, z = q / (G.nx * G.ny);
            T dv[3];
            lex_div(G, sm.e[s], sm.eta[s], x, y, z, dv);
            for (int c = 0; c < 3; c++) {
                size_t id = (size_t)c * n + q;
                sm.t[s][id] = sm.r[s][id] - sm.e[s][id] - coef * dv[c];
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < 3 * nc_; q += blockDim.x) {
            int c = q / nc_, cq = q % nc_;
            int x = cq % C.nx, y = (cq / C.nx) % C.ny, z = cq / (C.nx * C.ny);
            T acc = 0;
            for (int dk = 0; dk < 2; dk++)
                for (int dj = 0; dj < 2; dj++)
                    for (int di = 0; di < 2; di++) acc += sm.t[s][G.id(c, 2 * x + di, 2 * y + dj, 2 * z + dk)];
            sm.r[s + 1][q] = acc / T(8);
            sm.e[s + 1][q] = T(0);
        }
        __syncthreads();
    }
    lex_sweeps(sm, s, lamdt, nc);
    for (s = sm.n - 2; s >= 0; s--) {
        LexGrid<T> G{sm.dims[s][0], sm.dims[s][1], sm.dims[s][2]};
        LexGrid<T> C{sm.dims[s + 1][0], sm.dims[s + 1][1], sm.dims[s + 1][2]};
        const int n = G.nx * G.ny * G.nz;
        for (int q = threadIdx.x; q < 3 * n; q += blockDim.x) {
            int c = q / n, fq = q % n;
            int x = fq % G.nx, y = (fq / G.nx) % G.ny, z = fq / (G.nx * G.ny);
            int px = x >> 1, py = y >> 1, pz = z >> 1;
            int sx = (x & 1) ? 1 : -1, sy = (y & 1) ? 1 : -1, sz = (z & 1) ? 1 : -1;
            T v = 0;
            for (int ak = 0; ak < 2; ak++)
                for (int aj = 0; aj < 2; aj++)
                    for (int ai = 0; ai < 2; ai++) {
                        T wt = (ai ? T(0.25) : T(0.75)) * (aj ? T(0.25) : T(0.75)) * (ak ? T(0.25) : T(0.75));
                        v += wt * sm.e[s + 1][C.id(c, px + ai * sx, py + aj * sy, pz + ak * sz)];
                    }
            sm.e[s][q] += v;
        }
        __syncthreads();
        lex_sweeps(sm, s, lamdt, nu2);
    }
}

// The same V-cycle over the lexicographic grids (float32) with the grids held in shared memory: e, r, t and eta of every grid are staged once (r of the first grid
// and eta from global memory, e from zero), every pass of the cycle runs between two block
// barriers, and only e of the first grid is written back.  The point update is the fused sweeps'
// (face_pair flux divergence, Eqs. 8-10, and the relaxed diagonal formed from eta, Eqs. 21-23)
// through an accessor whose periodic neighbour offsets are formed once per cell.
struct LexAcc {
    const float *fB, *fE;
    int n;                    // cells of the grid (component stride)
    int xo[3], yo[3], zo[3];  // offsets of the cells at -1, 0, +1 along x, y, z (wrapped)
    template <int C, int DX, int DY, int DZ>
    __device__ __forceinline__ float B() const {
        return fB[C * n + zo[DZ + 1] + yo[DY + 1] + xo[DX + 1]];
    }
    template <int DX, int DY, int DZ>
    __device__ __forceinline__ float E() const {
        return fE[zo[DZ + 1] + yo[DY + 1] + xo[DX + 1]];
    }
};

struct LexDims {
    int nx, ny, nz;
    int lx, ly;  // log2 of nx, ny when every extent is a power of two (p2)
    bool p2;
    __device__ __forceinline__ int n() const { return nx * ny * nz; }
    __device__ __forceinline__ int id(int x, int y, int z) const { return (z * ny + y) * nx + x; }
    __device__ __forceinline__ void cell(int q, int &x, int &y, int &z) const {
        if (p2) {
            x = q & (nx - 1);
            y = (q >> lx) & (ny - 1);
            z = q >> (lx + ly);
        } else {
            const int t = q / nx;
            x = q - t * nx;
            z = t / ny;
            y = t - z * ny;
        }
    }
    __device__ __forceinline__ LexAcc acc(const float *B, const float *E, int x, int y, int z) const {
        LexAcc a;
        a.fB = B;
        a.fE = E;
        a.n = n();
        const int pl = nx * ny;
        a.xo[0] = x > 0 ? x - 1 : nx - 1;
        a.xo[1] = x;
        a.xo[2] = x + 1 < nx ? x + 1 : 0;
        a.yo[0] = (y > 0 ? y - 1 : ny - 1) * nx;
        a.yo[1] = y * nx;
        a.yo[2] = (y + 1 < ny ? y + 1 : 0) * nx;
        a.zo[0] = (z > 0 ? z - 1 : nz - 1) * pl;
        a.zo[1] = z * pl;
        a.zo[2] = (z + 1 < nz ? z + 1 : 0) * pl;
        return a;
    }
};

struct BottomSm {  // no default member initialisers: a __shared__ copy is filled by one thread
    int n;
    LexDims d[MAX_SMALL];
    int base[MAX_SMALL];          // float offset of grid s in shared memory: e[3n], r[3n], t[3n], eta[n]
    RbK<float> K[MAX_SMALL];      // update constants of grid s (the sweeps' relaxed diagonal, Eqs. 21-23)
};

// the i-th cell of colour `colour` ((x + y + z) & 1) of a power-of-two grid with at least 2
// cells along x
__device__ __forceinline__ void colour_cell(const LexDims &D, int i, int colour, int &x, int &y, int &z) {
    const int hx = D.lx - 1;
    y = (i >> hx) & (D.ny - 1);
    z = i >> (hx + D.ly);
    x = 2 * (i & ((1 << hx) - 1)) + ((y + z + colour) & 1);
}

// one colour pass of grid s (Jacobi within the colour): t = (r - L e) / den on the colour's cells,
// then e += t
__device__ __forceinline__ void bsm_colour(const BottomSm &P, float *sh, int s, int colour) {
    const LexDims D = P.d[s];
    const int n = D.n();
    float *e = sh + P.base[s], *r = e + 3 * n, *t = r + 3 * n, *E = t + 3 * n;
    const RbK<float> K = P.K[s];
    // power-of-two grids at least 2 cells wide in x enumerate the colour's cells; other grids
    // visit every cell and skip the other colour
    const bool half = D.p2 && D.nx >= 2;
    const int ncol = half ? n / 2 : n;
    for (int i = threadIdx.x; i < ncol; i += blockDim.x) {
        int x, y, z;
        if (half) {
            colour_cell(D, i, colour, x, y, z);
        } else {
            D.cell(i, x, y, z);
            if (((x + y + z) & 1) != colour) continue;
        }
        const int q = D.id(x, y, z);
        const LexAcc a = D.acc(e, E, x, y, z);
        float es[6], den[3], dv[3];
        rb_faces_den<float>(a, K, es, den);
        cell_divergence<float>(a, es, dv);
#pragma unroll
        for (int c = 0; c < 3; c++)
            t[c * n + q] = rb_relax(0.f, v_mad(K.ncoef, dv[c], v_sub(r[c * n + q], e[c * n + q])), den[c]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ncol; i += blockDim.x) {
        int x, y, z;
        if (half) {
            colour_cell(D, i, colour, x, y, z);
        } else {
            D.cell(i, x, y, z);
            if (((x + y + z) & 1) != colour) continue;
        }
        const int q = D.id(x, y, z);
#pragma unroll
        for (int c = 0; c < 3; c++) e[c * n + q] = v_add(e[c * n + q], t[c * n + q]);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_bottom_sm(SmallDev<float> sm_all, BottomSm P_arg, int nu1, int nu2, int nc) {
    if (sm_all.imask && !sm_all.imask[blockIdx.x]) return;
    extern __shared__ __align__(16) float sh[];
    // the grid table and this instance's global arrays in shared memory (indexed by grid below;
    // kernel parameters are only read at compile-time indices)
    __shared__ BottomSm P;
    if (threadIdx.x == 0) P = P_arg;
    // stage r of grid 0 and eta of every grid; e of grid 0 starts from zero
#pragma unroll
    for (int g = 0; g < MAX_SMALL; g++) {
        if (g >= P_arg.n) break;
        const int n = P_arg.d[g].n();
        float *e = sh + P_arg.base[g], *r = e + 3 * n, *E = r + 6 * n;
        const float *eta = sm_all.eta[g] + (size_t)blockIdx.x * n;
        for (int q = threadIdx.x; q < n; q += blockDim.x) E[q] = eta[q];
        if (g == 0) {
            const float *r0 = sm_all.r[0] + (size_t)blockIdx.x * 3 * n;
            for (int q = threadIdx.x; q < 3 * n; q += blockDim.x) {
                r[q] = r0[q];
                e[q] = 0.f;
            }
        }
    }
    __syncthreads();
    int s = 0;
    for (; s < P.n - 1; s++) {
        for (int k = 0; k < nu1; k++) {
            bsm_colour(P, sh, s, 0);
            bsm_colour(P, sh, s, 1);
        }
        const LexDims D = P.d[s], C = P.d[s + 1];
        const int n = D.n(), ncs = C.n();
        float *e = sh + P.base[s], *r = e + 3 * n, *t = r + 3 * n, *E = t + 3 * n;
        for (int q = threadIdx.x; q < n; q += blockDim.x) {  // residual t = r - L e
            int x, y, z;
            D.cell(q, x, y, z);
            const LexAcc a = D.acc(e, E, x, y, z);
            float es[6], dv[3];
            face_sums<float>(a, es);
            cell_divergence<float>(a, es, dv);
#pragma unroll
            for (int c = 0; c < 3; c++) t[c * n + q] = v_mad(P.K[s].ncoef, dv[c], v_sub(r[c * n + q], e[c * n + q]));
        }
        __syncthreads();
        float *ec = sh + P.base[s + 1], *rc = ec + 3 * ncs;
        for (int q = threadIdx.x; q < 3 * ncs; q += blockDim.x) {  // mean of the 8 children; e = 0
            const int c = q / ncs, cq = q - c * ncs;
            int x, y, z;
            C.cell(cq, x, y, z);
            float acc = 0.f;
            for (int dk = 0; dk < 2; dk++)
                for (int dj = 0; dj < 2; dj++)
                    for (int di = 0; di < 2; di++)
                        acc = v_add(acc, t[c * n + D.id(2 * x + di, 2 * y + dj, 2 * z + dk)]);
            rc[q] = v_mul(acc, 0.125f);
            ec[q] = 0.f;
        }
        __syncthreads();
    }
    for (int k = 0; k < nc; k++) {
        bsm_colour(P, sh, s, 0);
        bsm_colour(P, sh, s, 1);
    }
    for (s = P.n - 2; s >= 0; s--) {
        const LexDims D = P.d[s], C = P.d[s + 1];
        const int n = D.n(), ncs = C.n();
        float *e = sh + P.base[s];
        const float *ec = sh + P.base[s + 1];

        for (int q = threadIdx.x; q < 3 * n; q += blockDim.x) {  // trilinear prolongation (weights 3/4, 1/4)
            const int c = q / n, fq = q - c * n;
            int x, y, z;
            D.cell(fq, x, y, z);
            const int px = x >> 1, py = y >> 1, pz = z >> 1;
            const int sx = (x & 1) ? 1 : -1, sy = (y & 1) ? 1 : -1, sz = (z & 1) ? 1 : -1;
            float v = 0.f;
            for (int ak = 0; ak < 2; ak++)
                for (int aj = 0; aj < 2; aj++)
                    for (int ai = 0; ai < 2; ai++) {
                        const float wt = (ai ? 0.25f : 0.75f) * (aj ? 0.25f : 0.75f) * (ak ? 0.25f : 0.75f);
                        int cx = px + ai * sx, cy = py + aj * sy, cz = pz + ak * sz;  // periodic wrap
                        cx = cx < 0 ? cx + C.nx : (cx >= C.nx ? cx - C.nx : cx);
                        cy = cy < 0 ? cy + C.ny : (cy >= C.ny ? cy - C.ny : cy);
                        cz = cz < 0 ? cz + C.nz : (cz >= C.nz ? cz - C.nz : cz);
                        v = v_mad(wt, ec[c * ncs + C.id(cx, cy, cz)], v);
                    }
            e[q] = v_add(e[q], v);
        }
        __syncthreads();
        for (int k = 0; k < nu2; k++) {
            bsm_colour(P, sh, s, 0);
            bsm_colour(P, sh, s, 1);
        }
    }
    const int n0 = P.d[0].n();
    float *e0 = sm_all.e[0] + (size_t)blockIdx.x * 3 * n0;
    for (int q = threadIdx.x; q < 3 * n0; q += blockDim.x) e0[q] = sh[P.base[0] + q];
}

constexpr size_t BOTTOM_SMEM_MAX = 200 * 1024;

static int ilog2_exact(int v) {
    int l = 0;
    while ((1 << l) < v) l++;
    return (1 << l) == v ? l : -1;
}

// the shared-memory solver's grid table and its shared-memory bytes; false when the grids do
// not fit
static bool bottom_table(const SmallDev<float> &sm, double lamdt, BottomSm &P, size_t &bytes) {
    P.n = sm.n;
    size_t off = 0;
    for (int q = 0; q < sm.n; q++) {
        const int lx = ilog2_exact(sm.dims[q][0]), ly = ilog2_exact(sm.dims[q][1]), lz = ilog2_exact(sm.dims[q][2]);
        P.d[q] = LexDims{sm.dims[q][0], sm.dims[q][1], sm.dims[q][2], lx, ly, lx >= 0 && ly >= 0 && lz >= 0};
        P.base[q] = (int)off;
        P.K[q] = rb_constants<float>(lamdt, sm.h[q], sm.omega);
        off += 10 * (size_t)sm.dims[q][0] * sm.dims[q][1] * sm.dims[q][2];
        off = (off + 3) & ~(size_t)3;
    }
    bytes = off * sizeof(float);
    return bytes <= BOTTOM_SMEM_MAX;
}

bool bottom_in_shared(const SmallDev<float> &sm) {
    BottomSm P;
    size_t bytes = 0;
    return sm.n > 0 && bottom_table(sm, 1.0, P, bytes);
}

template <typename T>
cudaError_t launch_bottom(const SmallDev<T> &sm, double lamdt, int nu_pre, int nu_post, int n_coarse, cudaStream_t s) {
    if (sm.n == 0) return cudaSuccess;
    if constexpr (std::is_same<T, float>::value) {
        // shared-memory solver when the grids fit
        BottomSm P;
        size_t bytes = 0;
        if (bottom_table(sm, lamdt, P, bytes)) {
            static const bool attr =
                (cudaFuncSetAttribute(k_bottom_sm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BOTTOM_SMEM_MAX), true);
            (void)attr;
            k_bottom_sm<<<sm.ninst, 1024, bytes, s>>>(sm, P, nu_pre, nu_post, n_coarse);
            return cudaGetLastError();
        }
    }
    k_bottom<T><<<sm.ninst, 1024, 0, s>>>(sm, lamdt, nu_pre, nu_post, n_coarse);
    return cudaGetLastError();
}
template cudaError_t launch_bottom<double>(const SmallDev<double> &, double, int, int, int, cudaStream_t);
template cudaError_t launch_bottom<float>(const SmallDev<float> &, double, int, int, int, cudaStream_t);

// Lexicographic grids too large for the one-block solver, stepped by grid-wide launches over
// all instances (thread per instance and cell): the same arithmetic as k_bottom, one kernel per
// colour pass (e_in -> e_out, the other colour copied), per residual, per restriction and per
// prolongation.
template <typename T>
__device__ __forceinline__ bool lex_cell(const SmallDev<T> &sm, int s, size_t tid, int &q, int &cell) {
    const int n = sm.dims[s][0] * sm.dims[s][1] * sm.dims[s][2];
    if (tid >= (size_t)sm.ninst * n) return false;
    q = (int)(tid / n);
    cell = (int)(tid - (size_t)q * n);
    return !(sm.imask && !sm.imask[q]);
}

template <typename T>
__global__ void __launch_bounds__(256) k_lex_pass(SmallDev<T> sm, int s, double lamdt, int colour, int to_t) {
    int q, cell;
    if (!lex_cell(sm, s, blockIdx.x * (size_t)blockDim.x + threadIdx.x, q, cell)) return;
    const LexGrid<T> G{sm.dims[s][0], sm.dims[s][1], sm.dims[s][2]};
    const int n = G.nx * G.ny * G.nz;
    const size_t o3 = (size_t)q * 3 * n;
    const T *src = (to_t ? sm.e[s] : sm.t[s]) + o3;
    T *dst = (to_t ? sm.t[s] : sm.e[s]) + o3;
    const int x = cell % G.nx, y = (cell / G.nx) % G.ny, z = cell / (G.nx * G.ny);
    if (((x + y + z) & 1) != colour) {
        for (int c = 0; c < 3; c++) dst[(size_t)c * n + cell] = src[(size_t)c * n + cell];
        return;
    }
    const T coef = (T)(lamdt / (2.0 * sm.h[s] * sm.h[s]));
    const T *r = sm.r[s] + o3, *inv = sm.inv[s] + o3, *E = sm.eta[s] + (size_t)q * n;
    T dv[3];
    lex_div(G, src, E, x, y, z, dv);
    for (int c = 0; c < 3; c++) {
        const size_t id = (size_t)c * n + cell;
        const T d = (r[id] - src[id] - coef * dv[c]) * inv[id];
        dst[id] = src[id] + d;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_lex_resid(SmallDev<T> sm, int s, double lamdt) {
    int q, cell;
    if (!lex_cell(sm, s, blockIdx.x * (size_t)blockDim.x + threadIdx.x, q, cell)) return;
    const LexGrid<T> G{sm.dims[s][0], sm.dims[s][1], sm.dims[s][2]};
    const int n = G.nx * G.ny * G.nz;
    const size_t o3 = (size_t)q * 3 * n;
    const T coef = (T)(lamdt / (2.0 * sm.h[s] * sm.h[s]));
    const T *e = sm.e[s] + o3, *r = sm.r[s] + o3, *E = sm.eta[s] + (size_t)q * n;
    T *t = sm.t[s] + o3;
    const int x = cell % G.nx, y = (cell / G.nx) % G.ny, z = cell / (G.nx * G.ny);
    T dv[3];
    lex_div(G, e, E, x, y, z, dv);
    for (int c = 0; c < 3; c++) {
        const size_t id = (size_t)c * n + cell;
        t[id] = r[id] - e[id] - coef * dv[c];
    }
}

// r of grid s + 1 = mean of the 8 children of t on grid s; e of grid s + 1 = 0
template <typename T>
__global__ void __launch_bounds__(256) k_lex_restrict(SmallDev<T> sm, int s) {
    int q, cell;
    if (!lex_cell(sm, s + 1, blockIdx.x * (size_t)blockDim.x + threadIdx.x, q, cell)) return;
    const LexGrid<T> G{sm.dims[s][0], sm.dims[s][1], sm.dims[s][2]};
    const LexGrid<T> C{sm.dims[s + 1][0], sm.dims[s + 1][1], sm.dims[s + 1][2]};
    const int n = G.nx * G.ny * G.nz, nc_ = C.nx * C.ny * C.nz;
    const T *t = sm.t[s] + (size_t)q * 3 * n;
    const int x = cell % C.nx, y = (cell / C.nx) % C.ny, z = cell / (C.nx * C.ny);
    for (int c = 0; c < 3; c++) {
        T acc = 0;
        for (int dk = 0; dk < 2; dk++)
            for (int dj = 0; dj < 2; dj++)
                for (int di = 0; di < 2; di++) acc += t[G.id(c, 2 * x + di, 2 * y + dj, 2 * z + dk)];
        const size_t id = (size_t)q * 3 * nc_ + (size_t)c * nc_ + cell;
        sm.r[s + 1][id] = acc / T(8);
        sm.e[s + 1][id] = T(0);
    }
}

// e of grid s += trilinear interpolation of e of grid s + 1
template <typename T>
__global__ void __launch_bounds__(256) k_lex_prolong(SmallDev<T> sm, int s) {
    int q, cell;
    if (!lex_cell(sm, s, blockIdx.x * (size_t)blockDim.x + threadIdx.x, q, cell)) return;
    const LexGrid<T> G{sm.dims[s][0], sm.dims[s][1], sm.dims[s][2]};
    const LexGrid<T> C{sm.dims[s + 1][0], sm.dims[s + 1][1], sm.dims[s + 1][2]};
    const int n = G.nx * G.ny * G.nz, nc_ = C.nx * C.ny * C.nz;
    const T *ec = sm.e[s + 1] + (size_t)q * 3 * nc_;
    T *e = sm.e[s] + (size_t)q * 3 * n;
    const int x = cell % G.nx, y = (cell / G.nx) % G.ny, z = cell / (G.nx * G.ny);
    const int px = x >> 1, py = y >> 1, pz = z >> 1;
    const int sx = (x & 1) ? 1 : -1, sy = (y & 1) ? 1 : -1, sz = (z & 1) ? 1 : -1;
    for (int c = 0; c < 3; c++) {
        T v = 0;
        for (int ak = 0; ak < 2; ak++)
            for (int aj = 0; aj < 2; aj++)
                for (int ai = 0; ai < 2; ai++) {
                    T wt = (ai ? T(0.25) : T(0.75)) * (aj ? T(0.25) : T(0.75)) * (ak ? T(0.25) : T(0.75));
                    v += wt * ec[C.id(c, px + ai * sx, py + aj * sy, pz + ak * sz)];
                }
        e[(size_t)c * n + cell] += v;
    }
}

template <typename T>
static unsigned lex_grid(const SmallDev<T> &sm, int s) {
    const size_t n = (size_t)sm.ninst * sm.dims[s][0] * sm.dims[s][1] * sm.dims[s][2];
    return (unsigned)((n + 255) / 256);
}

template <typename T>
cudaError_t launch_lex_sweeps(const SmallDev<T> &sm, int s, double lamdt, int nsweep, cudaStream_t st) {
    for (int i = 0; i < nsweep; i++) {
        k_lex_pass<T><<<lex_grid(sm, s), 256, 0, st>>>(sm, s, lamdt, 0, 1);  // e -> t: red
        k_lex_pass<T><<<lex_grid(sm, s), 256, 0, st>>>(sm, s, lamdt, 1, 0);  // t -> e: black
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lex_resid_restrict(const SmallDev<T> &sm, int s, double lamdt, cudaStream_t st) {
    k_lex_resid<T><<<lex_grid(sm, s), 256, 0, st>>>(sm, s, lamdt);
    k_lex_restrict<T><<<lex_grid(sm, s + 1), 256, 0, st>>>(sm, s);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lex_prolong(const SmallDev<T> &sm, int s, cudaStream_t st) {
    k_lex_prolong<T><<<lex_grid(sm, s), 256, 0, st>>>(sm, s);
    return cudaGetLastError();
}
template cudaError_t launch_lex_sweeps<double>(const SmallDev<double> &, int, double, int, cudaStream_t);
template cudaError_t launch_lex_sweeps<float>(const SmallDev<float> &, int, double, int, cudaStream_t);
template cudaError_t launch_lex_resid_restrict<double>(const SmallDev<double> &, int, double, cudaStream_t);
template cudaError_t launch_lex_resid_restrict<float>(const SmallDev<float> &, int, double, cudaStream_t);
template cudaError_t launch_lex_prolong<double>(const SmallDev<double> &, int, cudaStream_t);
template cudaError_t launch_lex_prolong<float>(const SmallDev<float> &, int, cudaStream_t);

// eta chain over the small grids (optional) and their inverse diagonals
template <typename T>
__global__ void __launch_bounds__(1024) k_small_setup(SmallDev<T> sm_all, double lamdt, int eta_chain) {
    const SmallDev<T> sm = small_instance(sm_all);
    if (eta_chain) {
        for (int s = 1; s < sm.n; s++) {
            LexGrid<T> F{sm.dims[s - 1][0], sm.dims[s - 1][1], sm.dims[s - 1][2]};
            LexGrid<T> C{sm.dims[s][0], sm.dims[s][1], sm.dims[s][2]};
            const int nc_ = C.nx * C.ny * C.nz;
            for (int q = threadIdx.x; q < nc_; q += blockDim.x) {
                int x = q % C.nx, y = (q / C.nx) % C.ny, z = q / (C.nx * C.ny);
                T acc = 0;
                for (int dk = 0; dk < 2; dk++)
                    for (int dj = 0; dj < 2; dj++)
                        for (int di = 0; di < 2; di++) acc += sm.eta[s - 1][F.id(0, 2 * x + di, 2 * y + dj, 2 * z + dk)];
                sm.eta[s][q] = acc / T(8);
            }
            __syncthreads();
        }
    }
    for (int s = 0; s < sm.n; s++) {
        LexGrid<T> G{sm.dims[s][0], sm.dims[s][1], sm.dims[s][2]};
        const int n = G.nx * G.ny * G.nz;
        const double lh2 = lamdt / (sm.h[s] * sm.h[s]);
        const T *E = sm.eta[s];
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            int x = q % G.nx, y = (q / G.nx) % G.ny, z = q / (G.nx * G.ny);
            double e0 = (double)E[q];
            double sa[3] = {0.5 * (e0 + (double)E[G.id(0, x + 1, y, z)]) + 0.5 * (e0 + (double)E[G.id(0, x - 1, y, z)]),
                            0.5 * (e0 + (double)E[G.id(0, x, y + 1, z)]) + 0.5 * (e0 + (double)E[G.id(0, x, y - 1, z)]),
                            0.5 * (e0 + (double)E[G.id(0, x, y, z + 1)]) + 0.5 * (e0 + (double)E[G.id(0, x, y, z - 1)])};
            for (int c = 0; c < 3; c++) {
                double al = 0.0;
                for (int ax = 0; ax < 3; ax++)
                    if (ax != c) al += lh2 * sa[ax];
                sm.inv[s][(size_t)c * n + q] = (T)(sm.omega / (1.0 + al));
            }
        }
        __syncthreads();
    }
}

template <typename T>
cudaError_t launch_small_setup(const SmallDev<T> &sm, double lamdt, bool eta_chain, cudaStream_t s) {
    if (sm.n == 0) return cudaSuccess;
    k_small_setup<T><<<sm.ninst, 1024, 0, s>>>(sm, lamdt, eta_chain ? 1 : 0);
    return cudaGetLastError();
}
template cudaError_t launch_small_setup<double>(const SmallDev<double> &, double, bool, cudaStream_t);
template cudaError_t launch_small_setup<float>(const SmallDev<float> &, double, bool, cudaStream_t);

}  // namespace ohm
