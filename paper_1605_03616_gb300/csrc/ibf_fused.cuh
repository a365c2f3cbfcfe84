// Structured-form apply of the preliminary IBF with several butterfly levels
// fused per kernel (FP32 or FP64 SIMT).
//
// Structure used (Sec. 2.1 and Sec. 3).  Because every Chebyshev grid is the
// same grid z shifted and scaled, the Lagrange weight of a child grid point
// in its parent box is one of two universal real matrices,
//   M^B_t(g^{C_c}_s) = T_c[t][s] = M_t((2c-1)/4 + z_s/2),  c = child index,
// so an H block (eq. PIBF2) is diag * T_c * diag and a G block (eq. PIBF3) is
// diag * T_a^T * diag with phase diagonals.  Adjacent diagonals are merged at
// construction, leaving per level one phase table D[i][C][.] (i: X box of the
// level, C: Omega child box).  Per butterfly unit (two input pairs (i', 2j+c),
// two output pairs (2i'+a, j)):
//   H level:  y_a[t] = sum_c sum_s T_c[t][s] D_{a,c}[s] x_c[s]
//   G level:  y_a[t] = sum_c D_{a,c}[t] sum_s T_a[s][t] x_c[s]
// and the adjoint runs the conjugate transposes in reverse level order.
//
// Fusion.  Output pairs (i0 2^k + a, jb) of level l0+k depend only on the
// input pairs (i0, jb 2^k + m) of level l0, so a CTA loads those 2^k pairs
// (r complex x rhs tile each) into shared memory, runs the k levels in place
// -- the unit of step s joins the two positions that differ in bit s-1, and
// the output bit replaces the consumed input bit, so outputs end in
// bit-reversed order -- and writes the 2^k results.  Global Lambda buffers
// use i-major pair order p = i 2^(L-l) + j with element (p r + t) nc + col;
// the first launch expands g through V^0, the switch M^h is applied in the
// epilogue of the launch that ends at level h, and the last launch evaluates
// u through U^L.
#pragma once

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "ibf_internal.h"

namespace ibf {

template <typename Real>
struct FusedTraits {
    // threads per CTA cap; FP64 keeps more registers per thread
    static constexpr int kThreads = sizeof(Real) == 4 ? 512 : 256;
    // resident CTAs per SM the register budget is sized for
    static constexpr int kMinBlocks = sizeof(Real) == 4 ? 2 : 1;
};

template <typename Real>
struct CT;
template <>
struct CT<float> {
    typedef float2 T;
};
template <>
struct CT<double> {
    typedef double2 T;
};

enum { PRO_LAMBDA = 0, PRO_V = 1, PRO_UADJ = 2 };
enum { EPI_LAMBDA = 0, EPI_SWITCH = 1, EPI_U = 2, EPI_VADJ = 3 };

// Even/odd form of the transfer matrices.  The Chebyshev grid is symmetric
// (z_{r-1-t} = -z_t), so T_1 = J T_0 J with J the index reversal.  With
// P = (I+J)/2 and Q = (I-J)/2:
//   T_0 y0 + T_1 y1 = P T_0 (y0 + J y1) + Q T_0 (y0 - J y1)           (H form)
//   T_0^T x = e + f,  T_1^T x = J (e - f),  e = T_0^T P x, f = T_0^T Q x   (G form)
// Each needs r^2 real multiply-adds per complex vector pair instead of 2 r^2.
template <int RP>
struct EO {
    static constexpr int HR = (RP + 1) / 2;   // even rows (incl. the middle one)
    static constexpr int HQ = RP / 2;         // odd rows
};

// Constants of the transfer matrices, shared by every launch with this r.
template <typename Real, int RP>
struct FusedConsts {
    // Pm[s][t] = (T0[t][s] + T0[RP-1-t][s]) / 2 (t < HQ); Pm[s][mid] = T0[mid][s]
    // Qm[s][t] = (T0[t][s] - T0[RP-1-t][s]) / 2 (t < HQ)
    // (stored by input index s, so one step of the H form reads a contiguous run)
    // E[t][s]  = (T0[s][t] + T0[RP-1-s][t]) / 2 (s < HQ); E[t][mid] = T0[mid][t]
    // F[t][s]  = (T0[s][t] - T0[RP-1-s][t]) / 2 (s < HQ)
    Real Pm[RP][EO<RP>::HR];
    Real Qm[RP][EO<RP>::HQ > 0 ? EO<RP>::HQ : 1];
    Real E[RP][EO<RP>::HR];
    Real F[RP][EO<RP>::HQ > 0 ? EO<RP>::HQ : 1];
    // the same weights as (w, w) pairs: one packed two-lane multiply-add
    // applies a weight to the real and imaginary part at once
    typename CT<Real>::T Pm2[RP][EO<RP>::HR];
    typename CT<Real>::T Qm2[RP][EO<RP>::HQ > 0 ? EO<RP>::HQ : 1];
    typename CT<Real>::T E2[RP][EO<RP>::HR];
    typename CT<Real>::T F2[RP][EO<RP>::HQ > 0 ? EO<RP>::HQ : 1];
};

// The weights depend only on r, so every translation unit that launches the
// fused kernels keeps one copy per (precision, r) in constant memory, filled
// once per device by fused_upload_consts (plan or batch creation).
template <typename Real, int RP>
__constant__ FusedConsts<Real, RP> c_eo;

// One fused launch of one transform: k levels starting at l0.
struct FusedDesc {
    const void* D[kMaxFuse];     // phase table of step s at D[s-1]
    const void* in;              // Lambda at the launch's input level
    void* out;                   // Lambda at the launch's output level
    const void* vin;             // g (forward) or y (adjoint), N x ncols column-major
    void* vout;                  // u (forward) or g (adjoint)
    const void* Vs;
    const void* Us;
    const void* Ms;
    const int32_t* perm;
    const int32_t* off;
    int64_t N;
    int L, l0, k, nc, rt, pro, epi, kind;
};

template <typename Real, int RP>
struct FusedParams {
    FusedConsts<Real, RP> C;
    FusedDesc d;
};

// Elements of the shared-memory region after the Lambda tile: the staged
// phase tables of the k levels (per-unit stride 4r), reused by the epilogues
// for the switch blocks (padded stride r^2+1) and U^L rows, and by the
// prologue for the V^0 rows.
__host__ __device__ __forceinline__ size_t fused_region_elems(int k, int RP)
{
    const size_t G = (size_t)1 << k;
    const size_t tables = (size_t)k * (G / 2) * (4 * RP);
    const size_t mblocks = G * ((size_t)RP * RP + 1);
    return tables > mblocks ? tables : mblocks;
}

__device__ __forceinline__ int brevk(int v, int nbits)
{
    return nbits ? (int)(__brev((unsigned)v) >> (32 - nbits)) : 0;
}

template <typename C>
__device__ __forceinline__ C cz()
{
    C r;
    r.x = 0;
    r.y = 0;
    return r;
}
template <typename C>
__device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b)  // conj(a) * b
{
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.x * b.y - a.y * b.x;
    return r;
}
template <typename C>
__device__ __forceinline__ void cacc(C& a, C b)
{
    a.x += b.x;
    a.y += b.y;
}
// acc += a b and acc += conj(a) b as chains of fused multiply-adds (four
// instructions instead of a product and a sum)
template <typename C>
__device__ __forceinline__ void cmac(C& acc, C a, C b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
template <typename C>
__device__ __forceinline__ void cmacc(C& acc, C a, C b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
template <bool CONJ, typename C>
__device__ __forceinline__ void cmacx(C& acc, C a, C b)
{
    if (CONJ)
        cmacc(acc, a, b);
    else
        cmac(acc, a, b);
}

// Asynchronous global -> shared copy of one complex element (no register
// round trip); !valid writes zeros.  Completed by cp_async_wait() before the
// barrier that publishes the shared memory.
__device__ __forceinline__ void cp_async_elem(float2* dst, const float2* src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2* dst, const double2* src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Layout of a unit's staged phase table (4r elements).  The unit's four
// diagonals D_{a,c} (row ac = 2a + c) are stored as two interleaved pairs,
// [p][t][w], so that one 16-byte shared load returns the two entries that a
// level step uses together:
//   H levels (KIND 0): pairs (D_00, D_10) and (D_01, D_11)
//   G levels (KIND 1): pairs (D_00, D_01) and (D_10, D_11)
// In both kinds the forward and the adjoint steps then read pair 0 at index t
// and pair 1 at index r-1-t.  The unit stride 4r and every pair offset are
// even, so with a 16-byte aligned table region every pair is 16-byte aligned.
template <int RP, int KIND>
__host__ __device__ __forceinline__ int tab_off(int ac, int t)
{
    const int p = KIND == 0 ? (ac & 1) : (ac >> 1);
    const int w = KIND == 0 ? (ac >> 1) : (ac & 1);
    return p * 2 * RP + 2 * t + w;
}
// the pair at q: q[0] and q[1] (one 16-byte load in single precision)
__device__ __forceinline__ void ld_pair(const float2* q, float2& a, float2& b)
{
    const float4 v = *reinterpret_cast<const float4*>(q);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(const double2* q, double2& a, double2& b)
{
    a = q[0];
    b = q[1];
}

// Two-lane arithmetic on (re, im) pairs: Blackwell's packed FP32 instructions
// (one issue slot for both lanes) in single precision, per-component double
// operations otherwise.  Rounding is that of the per-component operations:
// a - b is b * (-1) + a rounded once, w * x + acc is one fused multiply-add.
__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p2fma(float2 w, float2 x, float2 acc) { return __ffma2_rn(w, x, acc); }
__device__ __forceinline__ double2 p2add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 p2sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 p2fma(double2 w, double2 x, double2 acc)
{
    return make_double2(fma(w.x, x.x, acc.x), fma(w.y, x.y, acc.y));
}

}  // namespace ibf

#include "ibf_tc.cuh"

namespace ibf {

// Asynchronous copies of the phase tables of a fused block into dsm: every
// unit of every fused level, [s-1][u] with per-unit stride 4r in the pair
// layout of tab_off (the CTA reads each entry once from global memory); one
// thread per (level, unit, a, c) row of r contiguous entries.  Completed by
// cp_async_wait().
template <typename Real, int RP, int KIND>
__device__ __forceinline__ void fused_stage_tables(const FusedDesc& P, int64_t i0, int64_t jb, int k,
                                                   typename CT<Real>::T* dsm)
{
    typedef typename CT<Real>::T cx;
    constexpr int DS = 4 * RP;
    const int L = P.L, l0 = P.l0;
    const int nunit = (1 << k) >> 1;
    const int rows_per_level = nunit * 4;
    for (int row = threadIdx.x; row < k * rows_per_level; row += blockDim.x) {
        const int st1 = row / rows_per_level;          // level s = st1 + 1 of the launch
        const int rr = row - st1 * rows_per_level;
        const int u = rr >> 2, ac = rr & 3;             // ac = a * 2 + c
        const int s = st1 + 1, bit = st1;
        const int p0 = ((u >> bit) << (bit + 1)) | (u & ((1 << bit) - 1));
        const int low = p0 & ((1 << bit) - 1);
        const int64_t ia = (i0 << s) + ((int64_t)brevk(low, bit) << 1) + (ac >> 1);
        const int64_t C = (((jb << (k - s)) + (p0 >> s)) << 1) + (ac & 1);
        const int64_t ldC = 1LL << (L - l0 - s + 1);
        const cx* src = (const cx*)P.D[st1] + (ia * ldC + C) * RP;
        cx* dst = dsm + (st1 * nunit + u) * DS + tab_off<RP, KIND>(ac, 0);
#pragma unroll
        for (int t = 0; t < RP; ++t) cp_async_elem(dst + 2 * t, src + t, true);
    }
}

// The k butterfly levels of one block, in place in shared memory: sm holds
// the 2^k positions of the Lambda tile (stride PS = r rt + 1), dsm the staged
// phase tables [s-1][u] (per-unit stride 4r, pair layout of tab_off).  Every
// level ends with a barrier.
template <typename Real, int RP, bool ADJ, int KIND, int RT>
__device__ __forceinline__ void fused_levels(const FusedConsts<Real, RP>& C, int k, int rt_run, int ncol,
                                             typename CT<Real>::T* sm, const typename CT<Real>::T* dsm)
{
    typedef typename CT<Real>::T cx;
    const int rt = RT ? RT : rt_run;
    const int PS = RP * rt + 1;
    const int G = 1 << k;
    constexpr int DS = 4 * RP;
    constexpr int HR = EO<RP>::HR, HQ = EO<RP>::HQ;
    constexpr bool ODD = RP & 1;
    const int nunit = G >> 1;
    // One thread per (unit, column) computes both outputs of the unit and
    // writes them over its two inputs.  H form (forward H levels, adjoint
    // G levels): out_a = P T_0 (y_a0 + J y_a1) + Q T_0 (y_a0 - J y_a1).
    // G form (forward G levels, adjoint H levels): both outputs share
    // e = T_0^T P x_q and f = T_0^T Q x_q.
    constexpr bool TD = (!ADJ && KIND == 1) || (ADJ && KIND == 0);
    for (int st = 0; st < k; ++st) {
        const int s = ADJ ? (k - st) : (st + 1);
        const int bit = s - 1;
        const cx* dl = dsm + (size_t)(s - 1) * nunit * DS;
        if (!TD) {
            for (int w = threadIdx.x; w < nunit * rt; w += blockDim.x) {
                const int c = w % rt, u = w / rt;
                if (c < ncol) {
                    const int p0 = ((u >> bit) << (bit + 1)) | (u & ((1 << bit) - 1));
                    const int p1 = p0 | (1 << bit);
                    const cx* x0p = sm + (p0 * PS + c);
                    const cx* x1p = sm + (p1 * PS + c);
                    const cx* du = dl + u * DS;
                    // output a uses D_{a,q} (forward H) or conj(D_{q,a}) (adjoint G):
                    // d_{aq} below, with (d00, d10) the pair at s2 and (d01, d11)
                    // the pair at r-1-s2 (tab_off: forward H pairs D_{0c}, D_{1c};
                    // adjoint G, a G-kind table, pairs D_{c0}, D_{c1})
                    const cx* pa = du;
                    const cx* pb = du + 2 * RP;
                    cx we0[HR], wo0[HQ > 0 ? HQ : 1], we1[HR], wo1[HQ > 0 ? HQ : 1];
#pragma unroll
                    for (int t = 0; t < HR; ++t) we0[t] = we1[t] = cz<cx>();
#pragma unroll
                    for (int t = 0; t < HQ; ++t) wo0[t] = wo1[t] = cz<cx>();
#pragma unroll
                    for (int s2 = 0; s2 < RP; ++s2) {
                        const cx xa = x0p[s2 * rt], xb = x1p[(RP - 1 - s2) * rt];
                        cx d00, d10, d01, d11;
                        ld_pair(pa + 2 * s2, d00, d10);
                        ld_pair(pb + 2 * (RP - 1 - s2), d01, d11);
                        const cx y00 = ADJ ? cmulc(d00, xa) : cmul(d00, xa);
                        const cx y01 = ADJ ? cmulc(d01, xb) : cmul(d01, xb);
                        const cx y10 = ADJ ? cmulc(d10, xa) : cmul(d10, xa);
                        const cx y11 = ADJ ? cmulc(d11, xb) : cmul(d11, xb);
                        const cx pv0 = p2add(y00, y01), mv0 = p2sub(y00, y01);
                        const cx pv1 = p2add(y10, y11), mv1 = p2sub(y10, y11);
#pragma unroll
                        for (int t = 0; t < HR; ++t) {
                            const cx pm = C.Pm2[s2][t];
                            we0[t] = p2fma(pm, pv0, we0[t]);
                            we1[t] = p2fma(pm, pv1, we1[t]);
                        }
#pragma unroll
                        for (int t = 0; t < HQ; ++t) {
                            const cx qm = C.Qm2[s2][t];
                            wo0[t] = p2fma(qm, mv0, wo0[t]);
                            wo1[t] = p2fma(qm, mv1, wo1[t]);
                        }
                    }
                    cx* o0 = sm + (p0 * PS + c);
                    cx* o1 = sm + (p1 * PS + c);
#pragma unroll
                    for (int t = 0; t < HQ; ++t) {
                        o0[t * rt] = p2add(we0[t], wo0[t]);
                        o0[(RP - 1 - t) * rt] = p2sub(we0[t], wo0[t]);
                        o1[t * rt] = p2add(we1[t], wo1[t]);
                        o1[(RP - 1 - t) * rt] = p2sub(we1[t], wo1[t]);
                    }
                    if (ODD) {
                        o0[HQ * rt] = we0[HQ];
                        o1[HQ * rt] = we1[HQ];
                    }
                }
            }
        } else {
            for (int w = threadIdx.x; w < nunit * rt; w += blockDim.x) {
                const int c = w % rt, u = w / rt;
                if (c < ncol) {
                    const int p0 = ((u >> bit) << (bit + 1)) | (u & ((1 << bit) - 1));
                    const int p1 = p0 | (1 << bit);
                    const cx* du = dl + u * DS;
                    // even and odd parts of both inputs (all reads before any write)
                    cx xe[2][HR], xo[2][HQ > 0 ? HQ : 1];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const cx* xp = sm + ((q ? p1 : p0) * PS + c);
#pragma unroll
                        for (int s2 = 0; s2 < HQ; ++s2) {
                            const cx lo = xp[s2 * rt], hi = xp[(RP - 1 - s2) * rt];
                            xe[q][s2] = p2add(lo, hi);
                            xo[q][s2] = p2sub(lo, hi);
                        }
                        if (ODD) xe[q][HQ] = xp[HQ * rt];
                    }
                    cx* o0 = sm + (p0 * PS + c);
                    cx* o1 = sm + (p1 * PS + c);
#pragma unroll
                    for (int t = 0; t < RP; ++t) {
                        cx a0 = cz<cx>(), a1 = cz<cx>();
                        // forward G: dA_q = D_{0,q}[t], dB_q = D_{1,q}[r-1-t];
                        // adjoint H (an H-kind table): dA_q = D_{q,0}[t], dB_q = D_{q,1}[r-1-t]
                        cx dA[2], dB[2];
                        ld_pair(du + 2 * t, dA[0], dA[1]);
                        ld_pair(du + 2 * RP + 2 * (RP - 1 - t), dB[0], dB[1]);
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            cx e = cz<cx>(), f = cz<cx>();
#pragma unroll
                            for (int s2 = 0; s2 < HR; ++s2) e = p2fma(C.E2[t][s2], xe[q][s2], e);
#pragma unroll
                            for (int s2 = 0; s2 < HQ; ++s2) f = p2fma(C.F2[t][s2], xo[q][s2], f);
                            // (T_0^T x_q)[t] and (T_1^T x_q)[RP-1-t]
                            const cx z0 = p2add(e, f), z1 = p2sub(e, f);
                            // forward G: output a uses D_{a,q}; adjoint H: output c uses conj(D_{q,c})
                            cmacx<ADJ>(a0, dA[q], z0);
                            cmacx<ADJ>(a1, dB[q], z1);
                        }
                        o0[t * rt] = a0;
                        o1[(RP - 1 - t) * rt] = a1;
                    }
                }
            }
        }
        __syncthreads();
    }
    
}

// KIND: 0 = H levels (1..h), 1 = G levels (h+1..L).  RT: the rhs tile width
// when it is known at compile time (32, the batched case), 0 otherwise.
template <typename Real, int RP, bool ADJ, int KIND, int RT, bool COH = false, bool TCL = false>
__device__ __forceinline__ void fused_body(const FusedConsts<Real, RP>& C, const FusedDesc& P, int64_t blk,
                                           unsigned char* smraw, TcCtx* tc = nullptr)
{
    typedef typename CT<Real>::T cx;
    cx* sm = reinterpret_cast<cx*>(smraw);

    const int k = P.k, L = P.L, l0 = P.l0;
    const int rt = RT ? RT : P.rt;
    // shared-memory stride between pair positions, padded by one element so
    // that threads walking positions hit different banks
    const int PS = RP * rt + 1;
    const int G = 1 << k;
    const int ntile = (P.nc + rt - 1) / rt;
    const int64_t grp = blk / ntile;
    const int tile = (int)(blk - grp * ntile);
    const int col0 = tile * rt;
    const int ncol = min(rt, P.nc - col0);
    const int nbj = L - l0 - k;                 // bits of jb
    const int64_t i0 = grp >> nbj;
    const int64_t jb = grp & ((1LL << nbj) - 1);
    const int64_t N = P.N;

    constexpr int DS = 4 * RP;   // per-unit stride of the staged tables (pair layout of tab_off)
    // The persistent form (COH) runs every item of one level kind through one
    // non-inlined body, so it compiles in only the prologues and epilogues a
    // chunk of its kind can have (fewer live registers, fewer spills): the
    // switch level h lies in [1, L-1] and no chunk spans it, so forward H
    // chunks start with V^0 or a tile and end with the switch or a tile,
    // forward G chunks end with U^L or a tile, adjoint G chunks start with
    // U^L* or a tile and end with the switch or a tile, and adjoint H chunks
    // end with V^0* or a tile.  The per-launch kernels keep every branch.
    constexpr bool HAS_PRO_V = !COH || (!ADJ && KIND == 0);
    constexpr bool HAS_PRO_UADJ = !COH || (ADJ && KIND == 1);
    constexpr bool HAS_EPI_SWITCH = !COH || (!ADJ && KIND == 0) || (ADJ && KIND == 1);
    constexpr bool HAS_EPI_U = !COH || (!ADJ && KIND == 1);
    constexpr bool HAS_EPI_VADJ = !COH || (ADJ && KIND == 0);
    cx* dsm = sm + (size_t)G * PS;
    // a Lambda tile read through asynchronous copies: the table copies go out
    // with it, one wait and one barrier for both
    // (g and the V^0 rows, read only, go the same way in every mode)
    // (the tables are read-only during a launch, so the persistent form, whose
    // tile loads bypass L1, issues them early too)
    const bool early = P.pro == PRO_LAMBDA || P.pro == PRO_V;
    if (early) fused_stage_tables<Real, RP, KIND>(P, i0, jb, k, dsm);

    // ---------------------------------------------------------------- load
    if (HAS_PRO_V && P.pro == PRO_V) {
        // forward, l0 = 0: Lambda^0_{0,j} = V^0-expansion of g(xi_j), j = jb 2^k + pos.
        // The block's g values ([c][pos]) and its V^0 rows (contiguous) are
        // staged after the table region, with the table copies in flight.
        cx* gt = dsm + fused_region_elems(k, RP);
        cx* vs = gt + (size_t)G * rt;
        const cx* g = (const cx*)P.vin + (jb << k);
        for (int e = threadIdx.x; e < G * rt; e += blockDim.x) {
            const int pos = e & (G - 1), c = e >> k;
            const bool on = c < ncol;
            cp_async_elem(gt + e, g + pos + N * (int64_t)(col0 + (on ? c : 0)), on);
        }
        const cx* Vg = (const cx*)P.Vs + (jb << k) * RP;
        for (int e = threadIdx.x; e < G * RP; e += blockDim.x) cp_async_elem(vs + e, Vg + e, true);
        cp_async_wait();
        __syncthreads();
        for (int e = threadIdx.x; e < G * rt; e += blockDim.x) {
            const int pos = e & (G - 1), c = e >> k;
            const cx gv = gt[e];
#pragma unroll
            for (int t = 0; t < RP; ++t) sm[pos * PS + t * rt + c] = cmul(vs[pos * RP + t], gv);
        }
    } else if (HAS_PRO_UADJ && P.pro == PRO_UADJ) {
        // adjoint, top level L: Lambda^L_i[t] = sum_{n in leaf i} conj(U[n][t]) y[perm n]
        const cx* y = (const cx*)P.vin;
        const cx* U = (const cx*)P.Us;
        for (int e = threadIdx.x; e < G * rt; e += blockDim.x) {
            const int il = e & (G - 1), c = e >> k;
            const int pos = brevk(il, k);
            const int64_t leaf = (i0 << k) + il;
            cx acc[RP];
#pragma unroll
            for (int t = 0; t < RP; ++t) acc[t] = cz<cx>();
            if (c < ncol) {
                const int32_t n1 = P.off[leaf + 1];
                for (int32_t n = P.off[leaf]; n < n1; ++n) {
                    const cx yv = y[P.perm[n] + N * (col0 + c)];
#pragma unroll
                    for (int t = 0; t < RP; ++t) cmacc(acc[t], U[(int64_t)n * RP + t], yv);
                }
            }
#pragma unroll
            for (int t = 0; t < RP; ++t) sm[pos * PS + t * rt + c] = acc[t];
        }
    } else {
        const cx* in = (const cx*)P.in;
        if (RT == 32) {
            // one warp per position: its r rows of 32 columns are copied
            // together (r copies in flight per lane); data written by other
            // CTAs of the same launch (COH) is read past L1 through registers
            const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
            const bool on = lane < ncol;
            for (int pos = threadIdx.x >> 5; pos < G; pos += nw) {
                const int64_t pair = !ADJ ? (i0 << (L - l0)) + (jb << k) + pos
                                          : (((i0 << k) + brevk(pos, k)) << nbj) + jb;
                // lanes past the last column copy nothing from column col0's (valid) row addresses
                const cx* src = in + pair * RP * P.nc + col0 + (on ? lane : 0);
                cx* dst = sm + pos * PS + lane;
                if (!COH) {
#pragma unroll
                    for (int t = 0; t < RP; ++t, src += P.nc) cp_async_elem(dst + t * 32, src, on);
                } else {
                    cx v[RP];
#pragma unroll
                    for (int t = 0; t < RP; ++t) v[t] = on ? __ldcg(src + (int64_t)t * P.nc) : cz<cx>();
#pragma unroll
                    for (int t = 0; t < RP; ++t) dst[t * 32] = v[t];
                }
            }
            cp_async_wait();
        } else {
            for (int e = threadIdx.x; e < G * RP * rt; e += blockDim.x) {
                const int c = e % rt, t = (e / rt) % RP, pos = e / (rt * RP);
                int64_t pair;
                if (!ADJ)
                    pair = (i0 << (L - l0)) + (jb << k) + pos;
                else
                    pair = (((i0 << k) + brevk(pos, k)) << nbj) + jb;
                const cx* a = in + (pair * RP + t) * P.nc + col0 + c;
                sm[pos * PS + t * rt + c] = c < ncol ? (COH ? __ldcg(a) : *a) : cz<cx>();
            }
        }
    }
    if (early) cp_async_wait();
    __syncthreads();

    // ------------------------------------------------- stage phase tables
    // (issued above together with the Lambda tile when the input is a tile)
    if (!early) {
        fused_stage_tables<Real, RP, KIND>(P, i0, jb, k, dsm);
        cp_async_wait();
        __syncthreads();
    }

    if constexpr (TCL) {
        // tensor-core G-form levels (forward G, adjoint H), FP32 only
        static_assert(sizeof(Real) == 4 && ((!ADJ && KIND == 1) || (ADJ && KIND == 0)), "G form, FP32");
        for (int st = 0; st < k; ++st) {
            const int s = ADJ ? (k - st) : (st + 1);
            tc_level_g<RP, ADJ, RT>(*tc, s - 1, G >> 1, rt, ncol, sm, dsm + (size_t)(s - 1) * (G >> 1) * DS);
            __syncthreads();
        }
    } else {
        fused_levels<Real, RP, ADJ, KIND, RT>(C, k, rt, ncol, sm, dsm);
    }

    // ---------------------------------------------------------------- store
    if (P.epi == EPI_LAMBDA) {
        cx* out = (cx*)P.out;
        if (RT == 32) {
            const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
            if (lane < ncol)
                for (int pos = threadIdx.x >> 5; pos < G; pos += nw) {
                    const int64_t pair = !ADJ ? (((i0 << k) + brevk(pos, k)) << nbj) + jb
                                              : (i0 << (L - l0)) + (jb << k) + pos;
                    cx* dst = out + pair * RP * P.nc + col0 + lane;
                    const cx* srcs = sm + pos * PS + lane;
#pragma unroll
                    for (int t = 0; t < RP; ++t, dst += P.nc) *dst = srcs[t * 32];
                }
        } else {
            for (int e = threadIdx.x; e < G * RP * rt; e += blockDim.x) {
                const int c = e % rt, t = (e / rt) % RP, pos = e / (rt * RP);
                if (c >= ncol) continue;
                int64_t pair;
                if (!ADJ)
                    pair = (((i0 << k) + brevk(pos, k)) << nbj) + jb;
                else
                    pair = (i0 << (L - l0)) + (jb << k) + pos;
                out[(pair * RP + t) * P.nc + col0 + c] = sm[pos * PS + t * rt + c];
            }
        }
    } else if (HAS_EPI_SWITCH && P.epi == EPI_SWITCH) {
        // forward: Lambda~ = M~' Lambda at level h; adjoint: Lambda = M~'^* Lambda~.
        // The CTA's G blocks of r x r are staged in the table region first.
        cx* out = (cx*)P.out;
        constexpr int MS = RP * RP + 1;   // padded block stride
        cx* msm = sm + (size_t)G * PS;
        {
            constexpr int BM = 8;
            const int total = G * RP * RP;
            for (int e0 = threadIdx.x; e0 < total; e0 += BM * blockDim.x) {
                cx v[BM];
#pragma unroll
                for (int b = 0; b < BM; ++b) {
                    const int e = e0 + b * blockDim.x;
                    if (e < total) {
                        const int pos = e / (RP * RP), rem = e - pos * (RP * RP);
                        const int64_t pair = !ADJ ? (((i0 << k) + brevk(pos, k)) << nbj) + jb
                                                  : (i0 << (L - l0)) + (jb << k) + pos;
                        v[b] = ((const cx*)P.Ms)[pair * RP * RP + rem];
                    }
                }
#pragma unroll
                for (int b = 0; b < BM; ++b) {
                    const int e = e0 + b * blockDim.x;
                    if (e < total) {
                        const int pos = e / (RP * RP), rem = e - pos * (RP * RP);
                        msm[pos * MS + rem] = v[b];
                    }
                }
            }
        }
        __syncthreads();
        if (RT == 32) {
            // two columns (c, c + 16) per thread: each staged weight feeds both
            for (int e = threadIdx.x; e < G * 16; e += blockDim.x) {
                const int c = e & 15, pos = e >> 4;
                const int64_t pair = !ADJ ? (((i0 << k) + brevk(pos, k)) << nbj) + jb
                                          : (i0 << (L - l0)) + (jb << k) + pos;
                cx xa[RP], xb[RP];
#pragma unroll
                for (int t = 0; t < RP; ++t) {
                    xa[t] = sm[pos * PS + t * 32 + c];
                    xb[t] = sm[pos * PS + t * 32 + c + 16];
                }
                const cx* Mp = msm + pos * MS;
                cx* oa = out + pair * RP * P.nc + col0 + c;
#pragma unroll
                for (int t = 0; t < RP; ++t) {
                    cx aa = cz<cx>(), ab = cz<cx>();
#pragma unroll
                    for (int s2 = 0; s2 < RP; ++s2) {
                        const cx mv = ADJ ? Mp[s2 * RP + t] : Mp[t * RP + s2];
                        cmacx<ADJ>(aa, mv, xa[s2]);
                        cmacx<ADJ>(ab, mv, xb[s2]);
                    }
                    if (c < ncol) oa[(int64_t)t * P.nc] = aa;
                    if (c + 16 < ncol) oa[(int64_t)t * P.nc + 16] = ab;
                }
            }
        } else
        for (int e = threadIdx.x; e < G * rt; e += blockDim.x) {
            const int c = e % rt, pos = e / rt;
            if (c >= ncol) continue;
            int64_t pair;
            if (!ADJ)
                pair = (((i0 << k) + brevk(pos, k)) << nbj) + jb;
            else
                pair = (i0 << (L - l0)) + (jb << k) + pos;
            cx x[RP];
#pragma unroll
            for (int t = 0; t < RP; ++t) x[t] = sm[pos * PS + t * rt + c];
            const cx* Mp = msm + pos * MS;
#pragma unroll
            for (int t = 0; t < RP; ++t) {
                cx acc = cz<cx>();
                if (!ADJ) {
#pragma unroll
                    for (int s2 = 0; s2 < RP; ++s2) cmac(acc, Mp[t * RP + s2], x[s2]);
                } else {
#pragma unroll
                    for (int s2 = 0; s2 < RP; ++s2) cmacc(acc, Mp[s2 * RP + t], x[s2]);
                }
                out[(pair * RP + t) * P.nc + col0 + c] = acc;
            }
        }
    } else if (HAS_EPI_U && P.epi == EPI_U) {
        // forward, level L: u(x_n) = sum_t U[n][t] Lambda^L_{leaf(n)}[t]
        cx* u = (cx*)P.vout;
        // the CTA's leaves are contiguous, so are their points [nb0, nb1);
        // their U rows are staged in the table region when they fit
        const int32_t nb0 = P.off[i0 << k], nb1 = P.off[(i0 + 1) << k];
        const bool staged = (int64_t)(nb1 - nb0) * RP <= (int64_t)fused_region_elems(k, RP);
        const cx* U = staged ? sm + (size_t)G * PS - (int64_t)nb0 * RP : (const cx*)P.Us;
        if (staged) {
            cx* us = sm + (size_t)G * PS;
            const cx* Ug = (const cx*)P.Us + (int64_t)nb0 * RP;
            for (int e = threadIdx.x; e < (nb1 - nb0) * RP; e += blockDim.x) us[e] = Ug[e];
            __syncthreads();
        }
        for (int e = threadIdx.x; e < G * rt; e += blockDim.x) {
            const int il = e & (G - 1), c = e >> k;
            if (c >= ncol) continue;
            const int pos = brevk(il, k);
            const int64_t leaf = (i0 << k) + il;
            cx x[RP];
#pragma unroll
            for (int t = 0; t < RP; ++t) x[t] = sm[pos * PS + t * rt + c];
            const int32_t n1 = P.off[leaf + 1];
            for (int32_t n = P.off[leaf]; n < n1; ++n) {
                cx acc = cz<cx>();
#pragma unroll
                for (int t = 0; t < RP; ++t) cmac(acc, U[(int64_t)n * RP + t], x[t]);
                u[P.perm[n] + N * (col0 + c)] = acc;
            }
        }
    } else if (HAS_EPI_VADJ) {
        // adjoint, level 0: g(xi_j) = sum_t conj(V[j][t]) Lambda^0_{0,j}[t]
        cx* g = (cx*)P.vout;
        const cx* V = (const cx*)P.Vs;
        for (int e = threadIdx.x; e < G * rt; e += blockDim.x) {
            const int pos = e & (G - 1), c = e >> k;
            if (c >= ncol) continue;
            const int64_t kx = (jb << k) + pos;
            cx acc = cz<cx>();
#pragma unroll
            for (int t = 0; t < RP; ++t) cmacc(acc, V[kx * RP + t], sm[pos * PS + t * rt + c]);
            g[kx + N * (col0 + c)] = acc;
        }
    }
}

// Single-transform launch.
template <typename Real, int RP, bool ADJ, int KIND, int RT>
__global__ void __launch_bounds__(FusedTraits<Real>::kThreads, FusedTraits<Real>::kMinBlocks)
    k_fused(const __grid_constant__ FusedParams<Real, RP> P)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    fused_body<Real, RP, ADJ, KIND, RT>(c_eo<Real, RP>, P.d, blockIdx.x, smraw);
}

// Single-transform launch with the G-form levels on the tensor cores (FP32
// tiles of 32 columns, 128 threads, 128 columns of tensor memory per CTA).
// The set-up and tear-down bracket the whole block; status receives 1 if a
// wait for the tensor cores expired.
template <int RP, bool ADJ, int KIND>
__global__ void __launch_bounds__(kTcThreads, 4)
    k_fused_tc(const __grid_constant__ FusedParams<float, RP> P, const __grid_constant__ TcOps B, int* status,
               int tail)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    TcCtx tc;
    tc_setup(tc, B, smraw + tail, status);
    fused_body<float, RP, ADJ, KIND, 32, false, true>(c_eo<float, RP>, P.d, blockIdx.x, smraw, &tc);
    tc_teardown(tc);
}

// Batched launch: CTA blocks [start[b], start[b+1]) run descriptor b, so one
// launch covers one fused chunk of many transforms of a batch whatever their
// sizes (all descriptors of a launch share the level kind and tile width).
template <typename Real, int RP, bool ADJ, int KIND, int RT>
__global__ void __launch_bounds__(FusedTraits<Real>::kThreads, FusedTraits<Real>::kMinBlocks)
    k_fused_batch(const __grid_constant__ FusedConsts<Real, RP> C, const FusedDesc* __restrict__ descs,
                  const int64_t* __restrict__ start, int n)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    int lo = 0, hi = n - 1;
    const int64_t b = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    fused_body<Real, RP, ADJ, KIND, RT>(c_eo<Real, RP>, descs[lo], b - start[lo], smraw);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Chunk {
    int lo, hi;   // levels lo+1 .. hi (forward direction)
    int kind;     // 0: H levels, 1: G levels
};

// split levels 1..h and h+1..L into balanced chunks of at most kmax levels
inline std::vector<Chunk> fused_schedule(int L, int h, int kmax)
{
    std::vector<Chunk> v;
    auto split = [&](int a, int b, int kind) {
        int n = b - a;
        int nch = (n + kmax - 1) / kmax;
        int lo = a;
        for (int c = 0; c < nch; ++c) {
            int len = n / nch + (c < n % nch ? 1 : 0);
            v.push_back({lo, lo + len, kind});
            lo += len;
        }
    };
    split(0, h, 0);
    split(h, L, 1);
    return v;
}

inline int pow2ceil(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// even/odd matrices of T_0 (see struct EO), from the plan's FP64 T_0
template <typename Real, int RP>
inline void fill_even_odd(const ibf_plan* p, FusedConsts<Real, RP>& C)
{
    constexpr int HQ = EO<RP>::HQ;
    const auto& T0 = p->T[0];
    for (int t = 0; t < HQ; ++t)
        for (int s = 0; s < RP; ++s) {
            C.Pm[s][t] = (Real)((T0[t][s] + T0[RP - 1 - t][s]) / 2);
            C.Qm[s][t] = (Real)((T0[t][s] - T0[RP - 1 - t][s]) / 2);
        }
    if (RP & 1)
        for (int s = 0; s < RP; ++s) C.Pm[s][HQ] = (Real)T0[HQ][s];
    for (int t = 0; t < RP; ++t) {
        for (int s = 0; s < HQ; ++s) {
            C.E[t][s] = (Real)((T0[s][t] + T0[RP - 1 - s][t]) / 2);
            C.F[t][s] = (Real)((T0[s][t] - T0[RP - 1 - s][t]) / 2);
        }
        if (RP & 1) C.E[t][HQ] = (Real)T0[HQ][t];
    }
    for (int s = 0; s < RP; ++s) {
        for (int t = 0; t < EO<RP>::HR; ++t) {
            C.Pm2[s][t].x = C.Pm2[s][t].y = C.Pm[s][t];
            C.E2[s][t].x = C.E2[s][t].y = C.E[s][t];
        }
        for (int t = 0; t < HQ; ++t) {
            C.Qm2[s][t].x = C.Qm2[s][t].y = C.Qm[s][t];
            C.F2[s][t].x = C.F2[s][t].y = C.F[s][t];
        }
    }
}

// copy the even/odd weights of r = RP into this translation unit's constant
// memory on the current device (idempotent; synchronous, so call it outside
// stream capture -- plan and batch creation do).  Static, not inline: each
// translation unit has its own copy of c_eo and so its own "done" flags.
template <typename Real, int RP>
static int fused_upload_consts_t(const ibf_plan* p)
{
    static bool done[64] = {false};
    static std::mutex mu;   // plans may be created from several host threads
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return IBF_OK;
    FusedConsts<Real, RP> h;
    memset(&h, 0, sizeof(h));
    fill_even_odd(p, h);
    cudaError_t e = cudaMemcpyToSymbol(c_eo<Real, RP>, &h, sizeof(h));
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyToSymbol(even/odd weights)");
    if (dev >= 0 && dev < 64) done[dev] = true;
    return IBF_OK;
}

template <typename Real>
static int fused_upload_consts(const ibf_plan* p)
{
    switch (p->r) {
    case 5: return fused_upload_consts_t<Real, 5>(p);
    case 7: return fused_upload_consts_t<Real, 7>(p);
    case 9: return fused_upload_consts_t<Real, 9>(p);
    case 11: return fused_upload_consts_t<Real, 11>(p);
    default: return IBF_OK;
    }
}

// dynamic shared memory of one fused CTA: the Lambda tile plus the staged
// phase tables of its k levels (per-unit stride 4r); a launch with
// the V^0 prologue also stages its g values and V^0 rows
inline size_t fused_smem_bytes(int k, int rt, int RP, size_t esz, int pro = PRO_LAMBDA)
{
    const size_t G = (size_t)1 << k;
    const size_t extra = pro == PRO_V ? G * ((size_t)rt + RP) : 0;
    return (G * ((size_t)RP * rt + 1) + fused_region_elems(k, RP) + extra) * esz;
}

// largest fusion depth whose CTA fits the shared-memory budget that keeps
// two CTAs per SM
inline int fused_kmax(int rt, int RP, size_t esz)
{
    const size_t budget = 100 * 1024;
    int k = 1;
    while (k < kMaxFuse && fused_smem_bytes(k + 1, rt, RP, esz) <= budget) ++k;
    return k;
}

template <typename Real, int RP, bool ADJ, int KIND, int RT>
static void set_smem_attr()
{
    static bool done = false;
    if (!done) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncSetAttribute(k_fused<Real, RP, ADJ, KIND, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        done = true;
    }
}

// shared memory of a tensor-core CTA: the fused tile and tables, then (at a
// 128-byte boundary) the B operands, the barrier and the tensor-memory address
inline size_t tc_tail_offset(int k, int RP) { return (fused_smem_bytes(k, 32, RP, sizeof(float2)) + 127) & ~(size_t)127; }
inline size_t tc_smem_bytes(int k, int RP) { return tc_tail_offset(k, RP) + sizeof(TcOps) + 16; }

template <int RP, bool ADJ, int KIND>
static void launch_tc(const FusedParams<float, RP>& P, const TcOps& B, int* status, int64_t blocks, cudaStream_t st)
{
    static bool attr_done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncSetAttribute(k_fused_tc<RP, ADJ, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    k_fused_tc<RP, ADJ, KIND><<<(unsigned)blocks, kTcThreads, tc_smem_bytes(P.d.k, RP), st>>>(
        P, B, status, (int)tc_tail_offset(P.d.k, RP));
}

template <typename Real, int RP, bool ADJ, int KIND>
static int launch_one(const FusedParams<Real, RP>& P, int64_t ngroups, cudaStream_t st, const TcOps* tcb = nullptr,
                      int* tcstatus = nullptr)
{
    typedef typename CT<Real>::T cx;
    const int G = 1 << P.d.k;
    if constexpr (sizeof(Real) == 4 && ((!ADJ && KIND == 1) || (ADJ && KIND == 0))) {
        if (tcb && P.d.rt == 32) {
            launch_tc<RP, ADJ, KIND>(P, *tcb, tcstatus, ngroups * ((P.d.nc + 31) / 32), st);
            return IBF_OK;
        }
    }
    size_t smem = fused_smem_bytes(P.d.k, P.d.rt, RP, sizeof(cx), P.d.pro);
    int ntile = (P.d.nc + P.d.rt - 1) / P.d.rt;
    int threads = std::min(FusedTraits<Real>::kThreads, std::max(32, (G / 2) * P.d.rt));
    threads = (threads + 31) / 32 * 32;
    int64_t blocks = ngroups * ntile;
    if (P.d.rt == 32) {
        set_smem_attr<Real, RP, ADJ, KIND, 32>();
        k_fused<Real, RP, ADJ, KIND, 32><<<(unsigned)blocks, threads, smem, st>>>(P);
    } else if (P.d.rt == 16 && sizeof(Real) == 4) {
        set_smem_attr<Real, RP, ADJ, KIND, 16>();
        k_fused<Real, RP, ADJ, KIND, 16><<<(unsigned)blocks, threads, smem, st>>>(P);
    } else {
        set_smem_attr<Real, RP, ADJ, KIND, 0>();
        k_fused<Real, RP, ADJ, KIND, 0><<<(unsigned)blocks, threads, smem, st>>>(P);
    }
    return IBF_OK;
}

template <typename Real, int RP>
static int fused_run(ibf_plan* p, const void* vin, void* vout, int nrhs, bool adj, cudaStream_t st)
{
    typedef typename CT<Real>::T cx;
    FusedParams<Real, RP> P;
    memset(&P, 0, sizeof(P));
    int urc = fused_upload_consts_t<Real, RP>(p);
    if (urc) return urc;
    P.d.Vs = p->sV;
    P.d.Us = p->sU;
    P.d.Ms = p->sM;
    P.d.perm = p->d_perm;
    P.d.off = p->d_off;
    P.d.N = p->N;
    P.d.L = p->L;
    const int64_t N = p->N;
    TcOps tcb;
    const bool use_tc = sizeof(Real) == 4 && p->dtype == IBF_C64_TF32X3;
    if (use_tc) tc_build_ops(p->T[0], p->T[1], RP, tcb);
    for (int c0 = 0; c0 < nrhs; c0 += p->max_nrhs) {
        const int nc = std::min(p->max_nrhs, nrhs - c0);
        const int rt = std::min(p->rtile, pow2ceil(nc));
        int kmax = p->user_kfuse ? p->kfuse : fused_kmax(rt, RP, sizeof(cx));
        kmax = std::max(1, std::min(kmax, kMaxFuse));
        std::vector<Chunk> sched = fused_schedule(p->L, p->h, kmax);
        P.d.nc = nc;
        P.d.rt = rt;
        P.d.vin = (const cx*)vin + N * c0;
        P.d.vout = (cx*)vout + N * c0;
        void* bufs[2] = {p->ws[0], p->ws[1]};
        int cur = 0;   // buffer holding the current Lambda
        const int nch = (int)sched.size();
        prof_start(p, st);
        for (int ci = 0; ci < nch; ++ci) {
            const Chunk ch = adj ? sched[nch - 1 - ci] : sched[ci];
            P.d.l0 = ch.lo;
            P.d.kind = ch.kind;
            P.d.k = ch.hi - ch.lo;
            for (int s = 1; s <= P.d.k; ++s) P.d.D[s - 1] = p->stab[ch.lo + s];
            for (int s = P.d.k; s < kMaxFuse; ++s) P.d.D[s] = nullptr;
            if (!adj) {
                P.d.pro = ch.lo == 0 ? PRO_V : PRO_LAMBDA;
                P.d.epi = ch.hi == p->L ? EPI_U : (ch.hi == p->h ? EPI_SWITCH : EPI_LAMBDA);
            } else {
                P.d.pro = ch.hi == p->L ? PRO_UADJ : PRO_LAMBDA;
                P.d.epi = ch.lo == 0 ? EPI_VADJ : (ch.lo == p->h ? EPI_SWITCH : EPI_LAMBDA);
            }
            P.d.in = bufs[cur];
            P.d.out = bufs[cur ^ 1];
            const int64_t ngroups = 1LL << (p->L - P.d.k);
            int rc;
            const TcOps* tb = use_tc ? &tcb : nullptr;
            if (!adj)
                rc = ch.kind == 0 ? launch_one<Real, RP, false, 0>(P, ngroups, st, tb, p->d_status)
                                  : launch_one<Real, RP, false, 1>(P, ngroups, st, tb, p->d_status);
            else
                rc = ch.kind == 0 ? launch_one<Real, RP, true, 0>(P, ngroups, st, tb, p->d_status)
                                  : launch_one<Real, RP, true, 1>(P, ngroups, st, tb, p->d_status);
            if (rc) return rc;
            prof_mark(p, st, ch.kind == 0 ? IBF_K_FUSED_H : IBF_K_FUSED_G);
            cur ^= 1;
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : cuda_error(e, "fused apply launch");
}

template <typename Real>
static int fused_apply_t(ibf_plan* p, const void* vin, void* vout, int nrhs, bool adj, cudaStream_t st)
{
    switch (p->r) {
    case 5: return fused_run<Real, 5>(p, vin, vout, nrhs, adj, st);
    case 7: return fused_run<Real, 7>(p, vin, vout, nrhs, adj, st);
    case 9: return fused_run<Real, 9>(p, vin, vout, nrhs, adj, st);
    case 11: return fused_run<Real, 11>(p, vin, vout, nrhs, adj, st);
    default: return set_error(IBF_ERR_UNSUPPORTED, "structured form: unsupported r");
    }
}

}  // namespace ibf
