// Explicit-form apply of the preliminary IBF (Sec. 3): the plain form.
//
// u = U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^1)^* (V^0)^* g, one kernel per
// factor.  Lambda^l_{i,j} (r complex per box pair and right-hand side) is kept
// in i-major pair order p = i 2^(L-l) + j at every level, element
// (p r + t) nc + col, so the switch's reordering (Sec. 3, step 4) is only a
// change of index arithmetic.  Each butterfly block maps
// Lambda^{l-1}_{i/2, 2j+c} to Lambda^l_{i,j} (eqs. PIBF2, PIBF3).
//
// The optimal form runs the same kernels with its compressed blocks: rank r0
// at every level after the sweep-out stage, and after the sweep-in stage a
// rank per level (r_out x r_in blocks, an r_g x r_h middle factor).
#include <algorithm>
#include <type_traits>

#include "ibf_internal.h"

namespace ibf {

// Kernels are templates on the complex type: double2 for FP64 plans, float2
// for FP32 plans (factors built in FP64, then stored in FP32).
template <typename cx> struct RealOf;
template <> struct RealOf<double2> { typedef double T; };
template <> struct RealOf<float2> { typedef float T; };

template <typename cx>
__device__ __forceinline__ cx cmk(typename RealOf<cx>::T re, typename RealOf<cx>::T im)
{
    cx o;
    o.x = re;
    o.y = im;
    return o;
}
template <typename cx>
__device__ __forceinline__ cx cmul(cx a, cx b) { return cmk<cx>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename cx>
__device__ __forceinline__ cx cmulc(cx a, cx b)  // conj(a) * b
{
    return cmk<cx>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename cx>
__device__ __forceinline__ void cadd(cx& a, cx b) { a.x += b.x; a.y += b.y; }

// Lambda^0[k][t][col] = V[k][t] g[k + N col]       ((V^0)^* g, eq. step2mv1)
template <typename cd>
__global__ void kx_init(const cd* V, const cd* g, cd* lam, int64_t N, int r, int nc)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * r * nc) return;
    int col = (int)(e % nc);
    int t = (int)((e / nc) % r);
    int64_t k = e / ((int64_t)nc * r);
    lam[e] = cmul(V[k * r + t], g[k + N * col]);
}

// g[k + N col] = sum_t conj(V[k][t]) Lambda^0[k][t][col]
template <typename cd>
__global__ void kx_init_adj(const cd* V, const cd* lam, cd* g, int64_t N, int r, int nc)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * nc) return;
    int64_t k = e % N;
    int col = (int)(e / N);
    cd acc = cmk<cd>(0, 0);
    for (int t = 0; t < r; ++t) cadd(acc, cmulc(V[k * r + t], lam[(k * r + t) * nc + col]));
    g[k + N * col] = acc;
}

// one butterfly level l: out pair p = (i,j) (rank ro) from in pairs
// (i/2, 2j+c) (rank ri) through the ro x ri blocks blk[p][c]
template <typename cd>
__global__ void kx_level(const cd* blk, const cd* in, cd* out, int L, int l, int ro, int ri, int nc, int64_t N)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * ro * nc) return;
    int col = (int)(e % nc);
    int t = (int)((e / nc) % ro);
    int64_t p = e / ((int64_t)nc * ro);
    int64_t nj = 1LL << (L - l);
    int64_t i = p >> (L - l), j = p & (nj - 1);
    int64_t q0 = (i >> 1) * (2 * nj) + 2 * j;
    cd acc = cmk<cd>(0, 0);
    for (int c = 0; c < 2; ++c) {
        const cd* row = blk + ((p * 2 + c) * ro + t) * ri;
        const cd* v = in + (q0 + c) * ri * nc + col;
        for (int s = 0; s < ri; ++s) cadd(acc, cmul(row[s], v[(int64_t)s * nc]));
    }
    out[e] = acc;
}

// adjoint of level l: in pair q = (i', C) at level l-1 gathers from the two
// out pairs (2i'+a, C/2) at level l with the conjugated blocks
template <typename cd>
__global__ void kx_level_adj(const cd* blk, const cd* out, cd* in, int L, int l, int ro, int ri, int nc,
                             int64_t N)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * ri * nc) return;
    int col = (int)(e % nc);
    int s = (int)((e / nc) % ri);
    int64_t q = e / ((int64_t)nc * ri);
    int64_t nC = 1LL << (L - l + 1), nj = nC >> 1;
    int64_t ip = q >> (L - l + 1), C = q & (nC - 1);
    int64_t j = C >> 1;
    int c = (int)(C & 1);
    cd acc = cmk<cd>(0, 0);
    for (int a = 0; a < 2; ++a) {
        int64_t p = (2 * ip + a) * nj + j;
        const cd* col_blk = blk + ((p * 2 + c) * ro) * ri + s;
        const cd* v = out + p * ro * nc + col;
        for (int t = 0; t < ro; ++t) cadd(acc, cmulc(col_blk[(int64_t)t * ri], v[(int64_t)t * nc]));
    }
    in[e] = acc;
}

// Warp-per-pair forms of the two level kernels above (same arithmetic, same
// outputs).  A level streams its blocks once (2 ro ri entries per pair) and
// reads two contiguous input pairs, so it should run at the HBM rate; one
// thread per output entry instead issues ri dependent loads per block row
// and stays latency-bound.  Here one warp owns one output pair: it copies the
// pair's blocks and, per tile of kXCT columns, its inputs into a shared-memory
// slice with asynchronous copies (every lane several in flight), then each
// lane computes outputs (t, col) of the tile from shared memory (block rows
// read as broadcasts, inputs by consecutive columns) and stores them
// coalesced.  Ranks up to kXRmax.
constexpr int kXWarps = 8;     // warps (pairs) per CTA
constexpr int kXCT = 8;        // columns per tile
constexpr int kXRmax = 16;
constexpr int kXMinCols = 4;   // fewer columns leave most lanes of a pair's warp idle

__device__ __forceinline__ void xcp(float2* d, const float2* s)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(d)), "l"(s)
                 : "memory");
}
__device__ __forceinline__ void xcp(double2* d, const double2* s)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(d)), "l"(s)
                 : "memory");
}
__device__ __forceinline__ void xcp_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// shared memory per warp: the two blocks (or the two gathered blocks of the
// adjoint) and one tile of two input pairs
template <typename cd>
constexpr size_t xslice_elems() { return 2 * kXRmax * kXRmax + 2 * kXRmax * kXCT; }

template <typename cd>
__global__ void __launch_bounds__(kXWarps * 32) kx_level_w(const cd* blk, const cd* in, cd* out, int L, int l, int ro,
                                                            int ri, int nc, int64_t N)
{
    extern __shared__ __align__(16) unsigned char xsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kXWarps + w;
    if (p >= N) return;
    cd* sb = reinterpret_cast<cd*>(xsm) + w * xslice_elems<cd>();   // [c][t][s]
    cd* sx = sb + 2 * kXRmax * kXRmax;                                // [c][s][col of tile]
    const int64_t nj = 1LL << (L - l);
    const int64_t i = p >> (L - l), j = p & (nj - 1);
    const int64_t q0 = (i >> 1) * (2 * nj) + 2 * j;
    const cd* bp = blk + p * 2 * ro * ri;
    const int nb = 2 * ro * ri;
    for (int e = lane; e < nb; e += 32) xcp(sb + e, bp + e);
    for (int c0 = 0; c0 < nc; c0 += kXCT) {
        const int nt = min(kXCT, nc - c0);
        const cd* xin = in + q0 * ri * nc + c0;
        for (int e = lane; e < 2 * ri * nt; e += 32) {
            const int cs = e / nt, col = e - cs * nt;   // cs = c ri + s
            xcp(sx + cs * kXCT + col, xin + (int64_t)cs * nc + col);
        }
        xcp_wait();
        __syncwarp();
        for (int o = lane; o < ro * nt; o += 32) {
            const int t = o / nt, col = o - t * nt;
            cd acc = cmk<cd>(0, 0);
            for (int c = 0; c < 2; ++c) {
                const cd* row = sb + (c * ro + t) * ri;
                const cd* v = sx + c * ri * kXCT + col;
#pragma unroll 4
                for (int s2 = 0; s2 < ri; ++s2) cadd(acc, cmul(row[s2], v[s2 * kXCT]));
            }
            out[(p * ro + t) * nc + c0 + col] = acc;
        }
        __syncwarp();   // the tile's inputs are read before the next tile's copies
    }
}

// adjoint of level l, warp per input pair q = (i', C) of level l-1: it
// gathers from the output pairs (2i'+a, C/2), a = 0, 1, through block c = C&1
// of each, conjugate-transposed
template <typename cd>
__global__ void __launch_bounds__(kXWarps * 32) kx_level_adj_w(const cd* blk, const cd* out, cd* in, int L, int l,
                                                                int ro, int ri, int nc, int64_t N)
{
    extern __shared__ __align__(16) unsigned char xsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * kXWarps + w;
    if (q >= N) return;
    cd* sb = reinterpret_cast<cd*>(xsm) + w * xslice_elems<cd>();   // [a][t][s]
    cd* sy = sb + 2 * kXRmax * kXRmax;                                // [a][t][col of tile]
    const int64_t nC = 1LL << (L - l + 1), nj = nC >> 1;
    const int64_t ip = q >> (L - l + 1), C = q & (nC - 1);
    const int64_t j = C >> 1;
    const int c = (int)(C & 1);
    const int nb = ro * ri;
    for (int a = 0; a < 2; ++a) {
        const int64_t pa = (2 * ip + a) * nj + j;
        const cd* bp = blk + (pa * 2 + c) * nb;
        for (int e = lane; e < nb; e += 32) xcp(sb + a * nb + e, bp + e);
    }
    for (int c0 = 0; c0 < nc; c0 += kXCT) {
        const int nt = min(kXCT, nc - c0);
        for (int a = 0; a < 2; ++a) {
            const int64_t pa = (2 * ip + a) * nj + j;
            const cd* yin = out + pa * ro * nc + c0;
            for (int e = lane; e < ro * nt; e += 32) {
                const int t = e / nt, col = e - t * nt;
                xcp(sy + (a * ro + t) * kXCT + col, yin + (int64_t)t * nc + col);
            }
        }
        xcp_wait();
        __syncwarp();
        for (int o = lane; o < ri * nt; o += 32) {
            const int s2 = o / nt, col = o - s2 * nt;
            cd acc = cmk<cd>(0, 0);
            for (int a = 0; a < 2; ++a) {
                const cd* bcol = sb + a * nb + s2;
                const cd* v = sy + a * ro * kXCT + col;
#pragma unroll 4
                for (int t = 0; t < ro; ++t) cadd(acc, cmulc(bcol[t * ri], v[t * kXCT]));
            }
            in[(q * ri + s2) * nc + c0 + col] = acc;
        }
        __syncwarp();
    }
}

// switch at level h: out_p = M~_p in_p (eq. switchlocM), M~_p of rows x cols
// (rank after x rank before the switch), or its adjoint
template <typename cd>
__global__ void kx_switch(const cd* M, const cd* in, cd* out, int rows, int cols, int nc, int64_t N, int adj)
{
    const int rout = adj ? cols : rows, rin = adj ? rows : cols;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * rout * nc) return;
    int col = (int)(e % nc);
    int t = (int)((e / nc) % rout);
    int64_t p = e / ((int64_t)nc * rout);
    const cd* Mp = M + p * rows * cols;
    const cd* v = in + p * rin * nc + col;
    cd acc = cmk<cd>(0, 0);
    if (!adj)
        for (int s = 0; s < cols; ++s) cadd(acc, cmul(Mp[t * cols + s], v[(int64_t)s * nc]));
    else
        for (int s = 0; s < rows; ++s) cadd(acc, cmulc(Mp[s * cols + t], v[(int64_t)s * nc]));
    out[e] = acc;
}

// u[perm[n] + nx col] = sum_t U[n][t] Lambda^L[leaf(n)][t][col]   (eq. PIBFbf3)
template <typename cd>
__global__ void kx_term(const cd* U, const int32_t* leaf, const int32_t* perm, const cd* lam, cd* u, int64_t nx,
                        int r, int nc)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nx * nc) return;
    int64_t n = e % nx;
    int col = (int)(e / nx);
    const cd* v = lam + (int64_t)leaf[n] * r * nc + col;
    cd acc = cmk<cd>(0, 0);
    for (int t = 0; t < r; ++t) cadd(acc, cmul(U[n * r + t], v[(int64_t)t * nc]));
    u[perm[n] + nx * col] = acc;
}

// Lambda^L[i][t][col] = sum_{n in leaf i} conj(U[n][t]) y[perm[n] + nx col]
template <typename cd>
__global__ void kx_term_adj(const cd* U, const int32_t* off, const int32_t* perm, const cd* y, cd* lam, int64_t N,
                            int64_t nx, int r, int nc)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * r * nc) return;
    int col = (int)(e % nc);
    int t = (int)((e / nc) % r);
    int64_t i = e / ((int64_t)nc * r);
    cd acc = cmk<cd>(0, 0);
    for (int32_t n = off[i]; n < off[i + 1]; ++n) cadd(acc, cmulc(U[(int64_t)n * r + t], y[perm[n] + nx * col]));
    lam[e] = acc;
}

static inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

// the warp-per-pair level kernels use kXWarps slices of shared memory (96 KB
// for complex128): raise their dynamic shared-memory limit once per device
template <typename cd>
static size_t xlevel_smem()
{
    static bool done[64] = {false};
    const size_t bytes = kXWarps * xslice_elems<cd>() * sizeof(cd);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !done[dev]) {
        cudaFuncSetAttribute(kx_level_w<cd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        cudaFuncSetAttribute(kx_level_adj_w<cd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (dev >= 0 && dev < 64) done[dev] = true;
    }
    return bytes;
}

// rank of Lambda^l before the switch (H side, l <= h) and after it (G side,
// l >= h)
static inline int rank_h(const ibf_plan* p, int l)
{
    return !p->rk_h.empty() ? p->rk_h[l] : (p->ra > 0 ? p->ra : p->r);
}
static inline int rank_g(const ibf_plan* p, int l)
{
    return !p->rk_g.empty() ? p->rk_g[l] : (p->ra > 0 ? p->ra : p->r);
}
// output and input rank of the butterfly blocks of level l
static inline int rank_out(const ibf_plan* p, int l) { return l <= p->h ? rank_h(p, l) : rank_g(p, l); }
static inline int rank_in(const ibf_plan* p, int l) { return l <= p->h ? rank_h(p, l - 1) : rank_g(p, l - 1); }

int explicit_launches(const ibf_plan* p) { return p->L + 3; }

// persistent warp-per-pair level: as many CTAs as are resident at once;
// false (nothing launched) if its slices do not fit one CTA's shared memory

// Bulk-copy pipeline form of the forward levels and the forward switch for
// complex64 plans with 4, 8, 12 or 16 columns.  A level streams every block
// once and reads each input pair twice (the two output pairs of a unit share
// it), so it is bound by HBM once enough bytes are in flight.  A persistent
// CTA (one per SM) walks chunks of B consecutive output pairs: their blocks
// are one contiguous run, and so are their input pairs (one run of pairs
// (i/2, 2j + c) per row, and rows 2i' and 2i'+1 share theirs; the switch
// reads pair p itself).  One producer lane copies each chunk with two
// cp.async.bulk transfers into a ring of shared-memory stages, completed on
// the stage's "full" mbarrier.  The consumer warps form groups of Gw warps,
// enough lanes for the chunk's B ro output rows; group g computes chunks g,
// g + ngroups, ... (one output row, all columns, per lane) and releases each
// stage on its "empty" mbarrier.  Each group owns sg stages of the ring and
// uses them in turn, so a stage has one consumer that sees its phases in
// order (a parity wait cannot tell phase n from phase n - 2), and the next
// chunk of every group is in flight while the group computes.  Every wait
// is bounded: when one expires the kernel sets *status, stops issuing copies,
// waits (bounded) for the copies it issued and returns.
constexpr int kXbWarps = 16;           // consumer warps per CTA
constexpr int kXbMaxStages = 16;
constexpr int kXbMaxPairs = 512;       // pairs per chunk
constexpr int kXbMaxGroupWarps = 4;    // warps per group: at least four groups
constexpr int kXbChunkBytes = 32 << 10;
constexpr int kXbSmemBudget = 200 << 10;

// Waits poll the barrier and sleep between polls, so that a waiting warp
// (the producer is usually ahead and waits for a free stage) takes few issue
// slots from the computing warps; at most kXbPolls polls, about 1 s in all
// before a wait counts as expired.
constexpr int kXbPolls = 1 << 22;
constexpr unsigned kXbSleepNs = 256;

__device__ __forceinline__ unsigned xb_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool xb_wait(unsigned mbar, unsigned parity)
{
    for (int i = 0; i < kXbPolls; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        __nanosleep(kXbSleepNs);
    }
    return false;
}

// one non-blocking check of a barrier phase
__device__ __forceinline__ bool xb_test(unsigned mbar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    return done != 0;
}

// first input pair of output pair p: (i/2, 2j) of level l-1 for a level, p
// itself for the switch
template <bool SW>
__device__ __forceinline__ int64_t xb_q0(int64_t p, int L, int l)
{
    if (SW) return p;
    const int64_t nj = 1LL << (L - l);
    return ((p >> (L - l)) >> 1) * (2 * nj) + 2 * (p & (nj - 1));
}

// One lane's outputs t = tq + m TQ (m < M, the last one stored only while
// t < ro) of one output pair in one column: bp points at row tq of block
// c = 0, xp at the lane's column of input pair c = 0 (inputs [c][s][col]), op
// at output (tq, col).  NC blocks per pair (2 for a level, 1 for the switch).
// Rows t >= ro of the last output read past the pair's blocks, at most TQ - 1
// rows, which stay inside the stage (its input run follows the blocks): the
// arithmetic runs unguarded and only the store is skipped.
// One output column (pair p, column col, all RO rows) of a level (NC = 2
// blocks) or the switch (NC = 1): u[t][col] = sum_c sum_s B_c[t][s] x_c[s][col].
// br points at block c = 0 of the pair ([c][t][s], blocks of RO x ri), xr at
// the lane's column of input pair c = 0 ([c][s][col], rows of nc columns),
// op at output (0, col).  The nc lanes of a pair read the same block entries
// (broadcasts) and consecutive input columns.
template <int RO, int NC>
__device__ __forceinline__ void xb_col(const float2* br, const float2* xr, float2* op, int ri, int nc)
{
    float2 acc[RO];
#pragma unroll
    for (int t = 0; t < RO; ++t) acc[t] = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float2* b = br + c * RO * ri;
        const float2* x = xr + c * ri * nc;
#pragma unroll 3
        for (int s2 = 0; s2 < ri; ++s2, ++b, x += nc) {
            const float2 xv = *x;
#pragma unroll
            for (int t = 0; t < RO; ++t) {
                const float2 bv = b[t * ri];
                acc[t].x = fmaf(bv.x, xv.x, acc[t].x);
                acc[t].x = fmaf(-bv.y, xv.y, acc[t].x);
                acc[t].y = fmaf(bv.x, xv.y, acc[t].y);
                acc[t].y = fmaf(bv.y, xv.x, acc[t].y);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < RO; ++t) op[(int64_t)t * nc] = acc[t];
}

// blk: NC RO x ri blocks per output pair, nc columns (2..32); chunks of B
// pairs; ngroups groups of Gw consumer warps (ngroups Gw <= kXbWarps) with sg
// stages each.  Chunk it of this CTA goes to group it % ngroups, as its chunk
// j = it / ngroups, in stage (it % ngroups) sg + j % sg, phase j / sg.
template <int RO, bool SW>
__global__ void __launch_bounds__((kXbWarps + 1) * 32, 1)
    kx_level_bulk(const float2* blk, const float2* in, float2* out, int L, int l, int ri, int nc, int64_t N, int B,
                  int Gw, int ngroups, int sg, int* status)
{
    constexpr int NC = SW ? 1 : 2;
    extern __shared__ __align__(16) unsigned char xsm[];
    __shared__ __align__(8) unsigned long long full[kXbMaxStages], empty[kXbMaxStages];
    __shared__ int s_abort;
    __shared__ long long s_nxt[kXbWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nb = NC * RO * ri;                                 // block entries per pair
    const size_t stage_elems = (size_t)B * nb + (size_t)NC * B * ri * nc;
    const int64_t nchunks = (N + B - 1) / B;
    const int stages = ngroups * sg;
    float2* sbase = reinterpret_cast<float2*>(xsm);
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(xb_smem(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(xb_smem(&empty[s])), "r"(Gw));
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (w == 0) {
        // producer: one lane issues the copies.  Each group's chunks go in the
        // group's order, but the groups are served independently: a round
        // visits every group and issues its next chunk if the stage it needs
        // is free, so a slow group does not hold up the others' copies.
        if (lane == 0) {
            long long* nxt = s_nxt;                     // next chunk (j) of each group
            for (int g = 0; g < ngroups; ++g) nxt[g] = 0;
            int idle = 0;
            bool left = true;
            while (left && !*(volatile int*)&s_abort) {
                left = false;
                bool issued = false;
                for (int g = 0; g < ngroups; ++g) {
                    const int64_t j = nxt[g];
                    const int64_t c = blockIdx.x + ((int64_t)g + j * ngroups) * gridDim.x;
                    if (c >= nchunks) continue;
                    left = true;
                    const int s = g * sg + (int)(j % sg);
                    const unsigned n = (unsigned)(j / sg);
                    if (n > 0 && !xb_test(xb_smem(&empty[s]), (n - 1) & 1)) continue;
                    const int64_t p0 = c * B;
                    const int64_t np = min((int64_t)B, N - p0);
                    const int64_t qlo = xb_q0<SW>(p0, L, l), qhi = xb_q0<SW>(p0 + np - 1, L, l) + NC;
                    const unsigned bb = (unsigned)(np * nb * sizeof(float2));
                    const unsigned ib = (unsigned)((qhi - qlo) * ri * nc * sizeof(float2));
                    float2* sb = sbase + (size_t)s * stage_elems;
                    const unsigned fb = xb_smem(&full[s]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(bb + ib)
                                 : "memory");
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
                            "r"(xb_smem(sb)),
                        "l"(blk + p0 * nb), "r"(bb), "r"(fb)
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
                            "r"(xb_smem(sb + (size_t)B * nb)),
                        "l"(in + qlo * ri * nc), "r"(ib), "r"(fb)
                        : "memory");
                    nxt[g] = j + 1;
                    issued = true;
                }
                if (left && !issued) {
                    if (++idle > kXbPolls) {
                        if (status) atomicExch(status, 1);
                        atomicExch(&s_abort, 1);
                        break;
                    }
                    __nanosleep(kXbSleepNs);
                } else {
                    idle = 0;
                }
            }
            // the last copies of every stage land before the CTA may exit
            for (int g = 0; g < ngroups; ++g)
                for (int64_t j = nxt[g] > sg ? nxt[g] - sg : 0; j < nxt[g]; ++j)
                    if (!xb_wait(xb_smem(&full[g * sg + (int)(j % sg)]), (unsigned)(j / sg) & 1) && status)
                        atomicExch(status, 1);
        }
        return;
    }
    // consumers: group g = (w - 1) / Gw computes chunks g, g + ngroups, ...;
    // a warp holds PW = 32 / nc pairs, nc lanes each (lane: one column); warp
    // gw of the group computes pairs gw PW + k, gw PW + k + Gw PW, ...
    const int g = (w - 1) / Gw, gw = (w - 1) - g * Gw;
    if (g >= ngroups) return;
    const int PW = 32 / nc, pk = lane / nc, col = lane - pk * nc;
    for (int64_t it = g, j = 0;; it += ngroups, ++j) {
        const int64_t c = blockIdx.x + it * gridDim.x;
        if (c >= nchunks) break;
        const int s = g * sg + (int)(j % sg);
        const unsigned n = (unsigned)(j / sg);
        if (!xb_wait(xb_smem(&full[s]), n & 1)) {
            if (status) atomicExch(status, 1);
            atomicExch(&s_abort, 1);
            break;
        }
        const int64_t p0 = c * B;
        const int64_t qlo = xb_q0<SW>(p0, L, l);
        const float2* sb = sbase + (size_t)s * stage_elems;
        const int np = (int)min((int64_t)B, N - p0);
        if (pk < PW)
            for (int b = gw * PW + pk; b < np; b += Gw * PW) {
                const int64_t p = p0 + b;
                xb_col<RO, NC>(sb + (size_t)b * nb, sb + (size_t)B * nb + (xb_q0<SW>(p, L, l) - qlo) * ri * nc + col,
                               out + p * RO * nc + col, ri, nc);
            }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(xb_smem(&empty[s])) : "memory");
        if (*(volatile int*)&s_abort) break;
    }
}

template <int RO, bool SW>
static bool launch_level_bulk_r(const float2* blk, const float2* in, float2* out, int L, int l, int ri, int nc,
                                int64_t N, int B, int Gw, int ngroups, int sg, size_t smem, int* status,
                                cudaStream_t st)
{
    int dev = 0, nsm = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the kernel's static shared memory (barriers, counters) is queried once per
    // device, and the dynamic limit raised to what remains of the opt-in size
    static size_t static_smem[64] = {0};
    if (dev < 0 || dev >= 64) return false;
    if (!static_smem[dev]) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, kx_level_bulk<RO, SW>) != cudaSuccess ||
            cudaFuncSetAttribute(kx_level_bulk<RO, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        static_smem[dev] = fa.sharedSizeBytes > 0 ? fa.sharedSizeBytes : 1;
    }
    if (smem + static_smem[dev] > (size_t)optin) return false;
    const int64_t blocks = std::min<int64_t>((N + B - 1) / B, (int64_t)nsm);
    kx_level_bulk<RO, SW><<<(unsigned)blocks, (kXbWarps + 1) * 32, smem, st>>>(blk, in, out, L, l, ri, nc, N, B, Gw,
                                                                                ngroups, sg, status);
    return true;
}

// Launch of kx_level_bulk for a level (SW false: two ro x ri blocks per
// output pair) or the forward switch (SW true: one block, input pair p), for
// 2..32 columns and ranks up to 16.  Chunks of B pairs (a power of two, at
// least 2, at most kXbMaxPairs) of at most kXbChunkBytes bytes; groups of
// Gw = min(ceil(B / PW), kXbMaxGroupWarps) warps (PW = 32 / nc pairs per warp,
// a lane loops over the chunk's pairs), each
// with two stages, as many groups as the warps and kXbSmemBudget allow.  One
// CTA per SM.  false when the shapes are outside its limits (then the caller
// runs another kernel).
template <bool SW>
static bool launch_level_bulk(const float2* blk, const float2* in, float2* out, int L, int l, int ro, int ri, int nc,
                              int64_t N, int* status, cudaStream_t st)
{
    if (nc < 2 || nc > 32 || ro < 1 || ri < 1 || ro > 16 || ri > 16 || N < 2) return false;
    const int NC = SW ? 1 : 2;
    const size_t pair_bytes = sizeof(float2) * ((size_t)NC * ro * ri + (size_t)NC * ri * nc);
    const int PW = 32 / nc;
    int B = 2;
    while (2 * B * pair_bytes <= (size_t)kXbChunkBytes && 2 * B <= N && 2 * B <= kXbMaxPairs) B *= 2;
    const int Gw = std::min((B + PW - 1) / PW, kXbMaxGroupWarps);
    if (Gw > kXbWarps) return false;
    const size_t stage_bytes = (size_t)B * pair_bytes;
    const int sg = 2;
    const int ngroups =
        (int)std::min<size_t>(kXbWarps / Gw, std::min<size_t>(kXbMaxStages, kXbSmemBudget / stage_bytes) / sg);
    if (ngroups < 1) return false;
    const size_t smem = (size_t)ngroups * sg * stage_bytes;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem + 1024 > (size_t)optin) return false;   // the kernel's own barriers and counters
#define XB_RO(R) \
    case R: return launch_level_bulk_r<R, SW>(blk, in, out, L, l, ri, nc, N, B, Gw, ngroups, sg, smem, status, st);
    switch (ro) {
        XB_RO(1) XB_RO(2) XB_RO(3) XB_RO(4) XB_RO(5) XB_RO(6) XB_RO(7) XB_RO(8)
        XB_RO(9) XB_RO(10) XB_RO(11) XB_RO(12) XB_RO(13) XB_RO(14) XB_RO(15) XB_RO(16)
    default: return false;
    }
#undef XB_RO
}

template <typename cd>
static int explicit_apply_t(ibf_plan* p, const void* gv, void* uv, int nrhs, cudaStream_t st)
{
    const int L = p->L, h = p->h;
    const int64_t N = p->N;
    const int k0 = rank_h(p, 0), kL = rank_g(p, L), mr = rank_g(p, h), mc = rank_h(p, h);
    for (int c0 = 0; c0 < nrhs; c0 += p->max_nrhs) {
        int nc = std::min(p->max_nrhs, nrhs - c0);
        const cd* g = (const cd*)gv + N * c0;
        cd* u = (cd*)uv + p->nx * c0;
        cd* a = (cd*)p->ws[0];
        cd* b = (cd*)p->ws[1];
        prof_start(p, st);
        kx_init<<<nb(N * k0 * nc), 256, 0, st>>>((const cd*)p->eV, g, a, N, k0, nc);
        prof_mark(p, st, IBF_K_EXPLICIT_INIT);
        for (int l = 1; l <= L; ++l) {
            const int ro = rank_out(p, l), ri = rank_in(p, l);
            // complex64 levels are memory-bound: the bulk-copy pipeline (up to 32
            // columns, ranks up to 16), else a warp per pair (more columns);
            // FP64 levels are bound by the FP64 pipe and keep one thread per
            // output entry, as do calls with fewer than kXMinCols columns
            const bool warp = sizeof(cd) == sizeof(float2) && nc >= kXMinCols;
            bool bulk = false;
            if constexpr (std::is_same<cd, float2>::value)
                bulk = warp && launch_level_bulk<false>((const float2*)p->eblk[l], a, b, L, l, ro, ri, nc, N,
                                                        p->d_status, st);
            if (bulk) {
            } else if (warp && ro <= kXRmax && ri <= kXRmax)
                kx_level_w<cd><<<(unsigned)((N + kXWarps - 1) / kXWarps), kXWarps * 32, xlevel_smem<cd>(), st>>>(
                    (const cd*)p->eblk[l], a, b, L, l, ro, ri, nc, N);
            else
                kx_level<<<nb(N * ro * nc), 256, 0, st>>>((const cd*)p->eblk[l], a, b, L, l, ro, ri, nc, N);
            prof_mark(p, st, IBF_K_EXPLICIT_LEVEL);
            std::swap(a, b);
            if (l == h) {
                bool bulk_sw = false;
                if constexpr (std::is_same<cd, float2>::value)
                    bulk_sw = nc >= kXMinCols && launch_level_bulk<true>((const float2*)p->eM, a, b, L, h, mr, mc, nc,
                                                                         N, p->d_status, st);
                if (!bulk_sw) kx_switch<<<nb(N * mr * nc), 256, 0, st>>>((const cd*)p->eM, a, b, mr, mc, nc, N, 0);
                prof_mark(p, st, IBF_K_EXPLICIT_SWITCH);
                std::swap(a, b);
            }
        }
        kx_term<<<nb(p->nx * nc), 256, 0, st>>>((const cd*)p->eU, p->d_leaf, p->d_perm, a, u, p->nx, kL, nc);
        prof_mark(p, st, IBF_K_EXPLICIT_TERM);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : cuda_error(e, "explicit apply launch");
}

template <typename cd>
static int explicit_adjoint_t(ibf_plan* p, const void* yv, void* gv, int nrhs, cudaStream_t st)
{
    const int L = p->L, h = p->h;
    const int64_t N = p->N;
    const int k0 = rank_h(p, 0), kL = rank_g(p, L), mr = rank_g(p, h), mc = rank_h(p, h);
    for (int c0 = 0; c0 < nrhs; c0 += p->max_nrhs) {
        int nc = std::min(p->max_nrhs, nrhs - c0);
        const cd* y = (const cd*)yv + p->nx * c0;
        cd* g = (cd*)gv + N * c0;
        cd* a = (cd*)p->ws[0];
        cd* b = (cd*)p->ws[1];
        prof_start(p, st);
        kx_term_adj<<<nb(N * kL * nc), 256, 0, st>>>((const cd*)p->eU, p->d_off, p->d_perm, y, a, N, p->nx, kL, nc);
        prof_mark(p, st, IBF_K_EXPLICIT_TERM);
        for (int l = L; l >= 1; --l) {
            if (l == h) {
                kx_switch<<<nb(N * mc * nc), 256, 0, st>>>((const cd*)p->eM, a, b, mr, mc, nc, N, 1);
                prof_mark(p, st, IBF_K_EXPLICIT_SWITCH);
                std::swap(a, b);
            }
            const int ro = rank_out(p, l), ri = rank_in(p, l);
            if (sizeof(cd) == sizeof(float2) && nc >= kXMinCols && ro <= kXRmax && ri <= kXRmax)
                kx_level_adj_w<cd><<<(unsigned)((N + kXWarps - 1) / kXWarps), kXWarps * 32, xlevel_smem<cd>(), st>>>(
                    (const cd*)p->eblk[l], a, b, L, l, ro, ri, nc, N);
            else
                kx_level_adj<<<nb(N * ri * nc), 256, 0, st>>>((const cd*)p->eblk[l], a, b, L, l, ro, ri, nc, N);
            prof_mark(p, st, IBF_K_EXPLICIT_LEVEL);
            std::swap(a, b);
        }
        kx_init_adj<<<nb(N * nc), 256, 0, st>>>((const cd*)p->eV, a, g, N, k0, nc);
        prof_mark(p, st, IBF_K_EXPLICIT_INIT);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : cuda_error(e, "explicit adjoint launch");
}

int explicit_apply(ibf_plan* p, const void* gv, void* uv, int nrhs, cudaStream_t st)
{
    return p->dtype == IBF_C128 ? explicit_apply_t<double2>(p, gv, uv, nrhs, st)
                                : explicit_apply_t<float2>(p, gv, uv, nrhs, st);
}

int explicit_adjoint(ibf_plan* p, const void* yv, void* gv, int nrhs, cudaStream_t st)
{
    return p->dtype == IBF_C128 ? explicit_adjoint_t<double2>(p, yv, gv, nrhs, st)
                                : explicit_adjoint_t<float2>(p, yv, gv, nrhs, st);
}

__global__ void kx_demote(const double2* a, float2* b, int64_t n)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// FP32 plans of the explicit and optimal forms: the factors are built (and
// compressed) in FP64, then replaced by complex64 copies.
int explicit_demote(ibf_plan* p, void* (*alloc)(ibf_plan*, size_t), void (*release)(ibf_plan*, void*))
{
    const int L = p->L, h = p->h;
    const int64_t N = p->N;
    auto one = [&](void*& f, int64_t n) -> int {
        void* q = alloc(p, sizeof(float2) * (size_t)n);
        if (!q) return set_error(IBF_ERR_OOM, "FP32 factor copy");
        kx_demote<<<nb(n), 256>>>((const double2*)f, (float2*)q, n);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_error(e, "FP32 factor copy");
        release(p, f);
        f = q;
        return IBF_OK;
    };
    int rc;
    if ((rc = one(p->eV, N * rank_h(p, 0)))) return rc;
    if ((rc = one(p->eM, N * rank_g(p, h) * rank_h(p, h)))) return rc;
    if ((rc = one(p->eU, p->nx * rank_g(p, L)))) return rc;
    for (int l = 1; l <= L; ++l)
        if ((rc = one(p->eblk[l], N * 2 * rank_out(p, l) * rank_in(p, l)))) return rc;
    p->factor_bytes = sizeof(float2) * (size_t)p->nnz;
    return IBF_OK;
}

}  // namespace ibf
