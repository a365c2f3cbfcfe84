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

template <typename Real, int RP>
struct FusedParams {
    Real T[2][RP][RP];           // T_c[t][s]; lives in the kernel parameter bank
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
    int L, l0, k, nc, rt, pro, epi;
};

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

// KIND: 0 = H levels (1..h), 1 = G levels (h+1..L).  RT: the rhs tile width
// when it is known at compile time (32, the batched case), 0 otherwise.
template <typename Real, int RP, bool ADJ, int KIND, int RT>
__global__ void __launch_bounds__(FusedTraits<Real>::kThreads, FusedTraits<Real>::kMinBlocks) k_fused(const __grid_constant__ FusedParams<Real, RP> P)
{
    typedef typename CT<Real>::T cx;
    extern __shared__ __align__(16) unsigned char smraw[];
    cx* sm = reinterpret_cast<cx*>(smraw);

    const int k = P.k, L = P.L, l0 = P.l0;
    const int rt = RT ? RT : P.rt;
    const int G = 1 << k;
    const int ntile = (P.nc + rt - 1) / rt;
    const int64_t grp = blockIdx.x / ntile;
    const int tile = blockIdx.x - (int)(grp * ntile);
    const int col0 = tile * rt;
    const int ncol = min(rt, P.nc - col0);
    const int nbj = L - l0 - k;                 // bits of jb
    const int64_t i0 = grp >> nbj;
    const int64_t jb = grp & ((1LL << nbj) - 1);
    const int64_t N = P.N;

    // ---------------------------------------------------------------- load
    if (P.pro == PRO_V) {
        // forward, l0 = 0: Lambda^0_{0,j} = V^0-expansion of g(xi_j), j = jb 2^k + pos
        const cx* g = (const cx*)P.vin;
        const cx* V = (const cx*)P.Vs;
        for (int e = threadIdx.x; e < G * rt; e += blockDim.x) {
            const int pos = e & (G - 1), c = e >> k;
            const int64_t kx = (jb << k) + pos;
            cx gv = c < ncol ? g[kx + N * (col0 + c)] : cz<cx>();
#pragma unroll
            for (int t = 0; t < RP; ++t) sm[(pos * RP + t) * rt + c] = cmul(V[kx * RP + t], gv);
        }
    } else if (P.pro == PRO_UADJ) {
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
                    for (int t = 0; t < RP; ++t) cacc(acc[t], cmulc(U[(int64_t)n * RP + t], yv));
                }
            }
#pragma unroll
            for (int t = 0; t < RP; ++t) sm[(pos * RP + t) * rt + c] = acc[t];
        }
    } else {
        const cx* in = (const cx*)P.in;
        for (int e = threadIdx.x; e < G * RP * rt; e += blockDim.x) {
            const int c = e % rt, t = (e / rt) % RP, pos = e / (rt * RP);
            int64_t pair;
            if (!ADJ)
                pair = (i0 << (L - l0)) + (jb << k) + pos;
            else
                pair = (((i0 << k) + brevk(pos, k)) << nbj) + jb;
            sm[e] = c < ncol ? in[(pair * RP + t) * P.nc + col0 + c] : cz<cx>();
        }
    }
    __syncthreads();

    // ------------------------------------------------- stage phase tables
    // D entries of every unit of every fused level, [s-1][u][a][c][RP]; the
    // CTA reads each once from global memory.
    constexpr int DS = 4 * RP + 1;   // per-unit stride, padded against bank conflicts
    cx* dsm = sm + (size_t)G * RP * rt;
    {
        const int nunit = G >> 1;
        const int per_level = nunit * 4 * RP;
        for (int st1 = 0; st1 < k; ++st1) {      // level s = st1 + 1 of the launch
            const int s = st1 + 1, bit = st1;
            const int64_t ldC = 1LL << (L - l0 - s + 1);
            const cx* Dg = (const cx*)P.D[st1];
            for (int e = threadIdx.x; e < per_level; e += blockDim.x) {
                const int u = e / (4 * RP);
                const int rem = e - u * (4 * RP);
                const int ac = rem / RP;                 // a * 2 + c
                const int t = rem - ac * RP;
                const int p0 = ((u >> bit) << (bit + 1)) | (u & ((1 << bit) - 1));
                const int low = p0 & ((1 << bit) - 1);
                const int64_t ia = (i0 << s) + ((int64_t)brevk(low, bit) << 1) + (ac >> 1);
                const int64_t C = (((jb << (k - s)) + (p0 >> s)) << 1) + (ac & 1);
                dsm[((size_t)st1 * nunit + u) * DS + rem] = __ldg(Dg + (ia * ldC + C) * RP + t);
            }
        }
    }
    __syncthreads();

    // --------------------------------------------------------------- levels
    // A warp owns UW units x CW columns; lanes 0-15 compute output 0 and
    // lanes 16-31 output 1 of the same (unit, column), so both inputs are read
    // before either output overwrites them (in place, __syncwarp between).
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
        const int o = lane >> 4, l16 = lane & 15;
        const int CW = rt < 16 ? rt : 16;
        const int UW = 16 / CW;
        const int nunit = G >> 1;
        const int nug = (nunit + UW - 1) / UW, nch = rt / CW;
        // TD forms use T_o^T; for o = 1 they run T_0^T on reversed vectors
        // (T_1 = J T_0 J for the symmetric Chebyshev grid), so the matrix
        // operand stays uniform across the warp.
        constexpr bool TD = (!ADJ && KIND == 1) || (ADJ && KIND == 0);
        for (int st = 0; st < k; ++st) {
            const int s = ADJ ? (k - st) : (st + 1);
            const int bit = s - 1;
            const cx* dl = dsm + (size_t)(s - 1) * nunit * DS;
            for (int task = warp; task < nug * nch; task += nwarp) {
                const int ug = task / nch, chn = task - ug * nch;
                const int u = ug * UW + l16 / CW;
                const int col = chn * CW + l16 % CW;
                const bool valid = u < nunit && col < ncol;
                const int uu = valid ? u : 0;
                const int p0 = ((uu >> bit) << (bit + 1)) | (uu & ((1 << bit) - 1));
                const int p1 = p0 | (1 << bit);
                const int cc = valid ? col : 0;
                const cx* x0p = sm + (size_t)p0 * RP * rt + cc;
                const cx* x1p = sm + (size_t)p1 * RP * rt + cc;
                const cx* du = dl + (size_t)uu * DS;
                cx acc[RP];
#pragma unroll
                for (int t = 0; t < RP; ++t) acc[t] = cz<cx>();
                if (!TD) {
                    // acc[t] = sum_q sum_s T_q[t][s] y_q[s],  y_q = D * x_q
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const cx* xp = q ? x1p : x0p;
                        const cx* dd = du + (ADJ ? (q * 2 + o) : (o * 2 + q)) * RP;
#pragma unroll
                        for (int s2 = 0; s2 < RP; ++s2) {
                            const cx xv = xp[s2 * rt];
                            const cx y = ADJ ? cmulc(dd[s2], xv) : cmul(dd[s2], xv);
#pragma unroll
                            for (int t = 0; t < RP; ++t) {
                                acc[t].x += P.T[q][t][s2] * y.x;
                                acc[t].y += P.T[q][t][s2] * y.y;
                            }
                        }
                    }
                } else {
                    // acc[t] = sum_q D[t] (T_o^T x_q)[t]; lanes with o = 1 walk
                    // x and D backwards (index RP-1-t) and use T_0
                    const int xstep = o ? -rt : rt;
                    const int dstep = o ? -1 : 1;
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const cx* xp = (q ? x1p : x0p) + (o ? (RP - 1) * rt : 0);
                        const cx* dd = du + (ADJ ? (q * 2 + o) : (o * 2 + q)) * RP + (o ? RP - 1 : 0);
                        cx xr[RP];
#pragma unroll
                        for (int s2 = 0; s2 < RP; ++s2) xr[s2] = xp[s2 * xstep];
#pragma unroll
                        for (int t = 0; t < RP; ++t) {
                            cx y = cz<cx>();
#pragma unroll
                            for (int s2 = 0; s2 < RP; ++s2) {
                                y.x += P.T[0][s2][t] * xr[s2].x;
                                y.y += P.T[0][s2][t] * xr[s2].y;
                            }
                            const cx dv = dd[t * dstep];
                            cacc(acc[t], ADJ ? cmulc(dv, y) : cmul(dv, y));
                        }
                    }
                }
                __syncwarp();
                if (valid) {
                    if (TD) {
                        cx* dst = sm + (size_t)(o ? p1 : p0) * RP * rt + col + (o ? (RP - 1) * rt : 0);
                        const int step = o ? -rt : rt;
#pragma unroll
                        for (int t = 0; t < RP; ++t) dst[t * step] = acc[t];
                    } else {
                        cx* dst = sm + (size_t)(o ? p1 : p0) * RP * rt + col;
#pragma unroll
                        for (int t = 0; t < RP; ++t) dst[t * rt] = acc[t];
                    }
                }
                __syncwarp();
            }
            __syncthreads();
        }
    }

    // ---------------------------------------------------------------- store
    if (P.epi == EPI_LAMBDA) {
        cx* out = (cx*)P.out;
        for (int e = threadIdx.x; e < G * RP * rt; e += blockDim.x) {
            const int c = e % rt, t = (e / rt) % RP, pos = e / (rt * RP);
            if (c >= ncol) continue;
            int64_t pair;
            if (!ADJ)
                pair = (((i0 << k) + brevk(pos, k)) << nbj) + jb;
            else
                pair = (i0 << (L - l0)) + (jb << k) + pos;
            out[(pair * RP + t) * P.nc + col0 + c] = sm[e];
        }
    } else if (P.epi == EPI_SWITCH) {
        // forward: Lambda~ = M~' Lambda at level h; adjoint: Lambda = M~'^* Lambda~
        cx* out = (cx*)P.out;
        const cx* M = (const cx*)P.Ms;
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
            for (int t = 0; t < RP; ++t) x[t] = sm[(pos * RP + t) * rt + c];
            const cx* Mp = M + pair * RP * RP;
#pragma unroll
            for (int t = 0; t < RP; ++t) {
                cx acc = cz<cx>();
                if (!ADJ) {
#pragma unroll
                    for (int s2 = 0; s2 < RP; ++s2) cacc(acc, cmul(__ldg(Mp + t * RP + s2), x[s2]));
                } else {
#pragma unroll
                    for (int s2 = 0; s2 < RP; ++s2) cacc(acc, cmulc(__ldg(Mp + s2 * RP + t), x[s2]));
                }
                out[(pair * RP + t) * P.nc + col0 + c] = acc;
            }
        }
    } else if (P.epi == EPI_U) {
        // forward, level L: u(x_n) = sum_t U[n][t] Lambda^L_{leaf(n)}[t]
        cx* u = (cx*)P.vout;
        const cx* U = (const cx*)P.Us;
        for (int e = threadIdx.x; e < G * rt; e += blockDim.x) {
            const int il = e & (G - 1), c = e >> k;
            if (c >= ncol) continue;
            const int pos = brevk(il, k);
            const int64_t leaf = (i0 << k) + il;
            cx x[RP];
#pragma unroll
            for (int t = 0; t < RP; ++t) x[t] = sm[(pos * RP + t) * rt + c];
            const int32_t n1 = P.off[leaf + 1];
            for (int32_t n = P.off[leaf]; n < n1; ++n) {
                cx acc = cz<cx>();
#pragma unroll
                for (int t = 0; t < RP; ++t) cacc(acc, cmul(U[(int64_t)n * RP + t], x[t]));
                u[P.perm[n] + N * (col0 + c)] = acc;
            }
        }
    } else {
        // adjoint, level 0: g(xi_j) = sum_t conj(V[j][t]) Lambda^0_{0,j}[t]
        cx* g = (cx*)P.vout;
        const cx* V = (const cx*)P.Vs;
        for (int e = threadIdx.x; e < G * rt; e += blockDim.x) {
            const int pos = e & (G - 1), c = e >> k;
            if (c >= ncol) continue;
            const int64_t kx = (jb << k) + pos;
            cx acc = cz<cx>();
#pragma unroll
            for (int t = 0; t < RP; ++t) cacc(acc, cmulc(V[kx * RP + t], sm[(pos * RP + t) * rt + c]));
            g[kx + N * (col0 + c)] = acc;
        }
    }
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

// dynamic shared memory of one fused CTA: the Lambda tile plus the staged
// phase tables of its k levels (padded per-unit stride 4r+1)
inline size_t fused_smem_bytes(int k, int rt, int RP, size_t esz)
{
    const size_t G = (size_t)1 << k;
    return (G * RP * rt + (size_t)k * (G / 2) * (4 * RP + 1)) * esz;
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

template <typename Real, int RP, bool ADJ, int KIND>
static int launch_one(const FusedParams<Real, RP>& P, int64_t ngroups, cudaStream_t st)
{
    typedef typename CT<Real>::T cx;
    const int G = 1 << P.k;
    size_t smem = fused_smem_bytes(P.k, P.rt, RP, sizeof(cx));
    int ntile = (P.nc + P.rt - 1) / P.rt;
    int threads = std::min(FusedTraits<Real>::kThreads, std::max(32, G * P.rt));
    threads = (threads + 31) / 32 * 32;
    int64_t blocks = ngroups * ntile;
    if (P.rt == 32) {
        set_smem_attr<Real, RP, ADJ, KIND, 32>();
        k_fused<Real, RP, ADJ, KIND, 32><<<(unsigned)blocks, threads, smem, st>>>(P);
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
    for (int c = 0; c < 2; ++c)
        for (int t = 0; t < RP; ++t)
            for (int s = 0; s < RP; ++s) P.T[c][t][s] = (Real)p->T[c][t][s];
    P.Vs = p->sV;
    P.Us = p->sU;
    P.Ms = p->sM;
    P.perm = p->d_perm;
    P.off = p->d_off;
    P.N = p->N;
    P.L = p->L;
    const int64_t N = p->N;
    for (int c0 = 0; c0 < nrhs; c0 += p->max_nrhs) {
        const int nc = std::min(p->max_nrhs, nrhs - c0);
        const int rt = std::min(p->rtile, pow2ceil(nc));
        int kmax = p->user_kfuse ? p->kfuse : fused_kmax(rt, RP, sizeof(cx));
        kmax = std::max(1, std::min(kmax, kMaxFuse));
        std::vector<Chunk> sched = fused_schedule(p->L, p->h, kmax);
        P.nc = nc;
        P.rt = rt;
        P.vin = (const cx*)vin + N * c0;
        P.vout = (cx*)vout + N * c0;
        void* bufs[2] = {p->ws[0], p->ws[1]};
        int cur = 0;   // buffer holding the current Lambda
        const int nch = (int)sched.size();
        prof_start(p, st);
        for (int ci = 0; ci < nch; ++ci) {
            const Chunk ch = adj ? sched[nch - 1 - ci] : sched[ci];
            P.l0 = ch.lo;
            P.k = ch.hi - ch.lo;
            for (int s = 1; s <= P.k; ++s) P.D[s - 1] = p->stab[ch.lo + s];
            for (int s = P.k; s < kMaxFuse; ++s) P.D[s] = nullptr;
            if (!adj) {
                P.pro = ch.lo == 0 ? PRO_V : PRO_LAMBDA;
                P.epi = ch.hi == p->L ? EPI_U : (ch.hi == p->h ? EPI_SWITCH : EPI_LAMBDA);
            } else {
                P.pro = ch.hi == p->L ? PRO_UADJ : PRO_LAMBDA;
                P.epi = ch.lo == 0 ? EPI_VADJ : (ch.lo == p->h ? EPI_SWITCH : EPI_LAMBDA);
            }
            P.in = bufs[cur];
            P.out = bufs[cur ^ 1];
            const int64_t ngroups = 1LL << (p->L - P.k);
            int rc;
            if (!adj)
                rc = ch.kind == 0 ? launch_one<Real, RP, false, 0>(P, ngroups, st)
                                  : launch_one<Real, RP, false, 1>(P, ngroups, st);
            else
                rc = ch.kind == 0 ? launch_one<Real, RP, true, 0>(P, ngroups, st)
                                  : launch_one<Real, RP, true, 1>(P, ngroups, st);
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
