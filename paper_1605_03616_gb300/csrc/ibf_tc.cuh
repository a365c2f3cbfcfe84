// Tensor-core (tcgen05) transfer products for the G form of a butterfly
// level (forward G levels; adjoint H levels have the same shape).
//
// In the G form both outputs of a unit share the transfer of each input:
//   z_{q,a}[t] = sum_s T_a[s][t] x_q[s]            (a, q in {0, 1}; Sec. 2.1's
//   out_a[t]   = sum_q D_{a,q}[t] z_{q,a}[t]        Lagrange transfer, eq. PIBF3)
// so the real matrix [T_0^T ; T_1^T] (2r x r) multiplies every input vector
// x_q of every (unit, column): one GEMM per level whose rows are the real and
// imaginary parts of the inputs, with a B operand shared by the whole launch.
// It runs on the 5th-generation tensor cores: the rows go from registers to
// tensor memory (tcgen05.st), one thread issues kind::tf32 MMAs with A in
// tensor memory and B in shared memory, the FP32 accumulators come back with
// tcgen05.ld, and the phase diagonals D are applied in FP32 SIMT arithmetic.
//
// Precision.  TF32 keeps 11 significant bits, so each operand is split in two
// TF32 terms: x = x_hi + x_lo (Veltkamp split with 2^13 + 1, exact in FP32;
// the tensor core truncates x_lo to 11 bits, an error below 2^-23 |x|) and
// w = w_hi + w_lo (rounded on the host from the FP64 T_c).  Three products
// are kept, x_hi w_hi + x_lo w_hi + x_hi w_lo; the dropped x_lo w_lo is below
// 2^-22 |x w|.  The K layout of one row of A is [x_hi (r) | x_lo (r) | 0 ...],
// product set 1 multiplies its first 24 columns by B1 = [w_hi ; w_hi ; 0] and
// set 2 its first 16 by B2 = [w_lo ; 0]: 3 + 2 MMAs of K = 8, N = 32 (the
// outputs of child a at columns 16 a + t).
#pragma once

#include <stdint.h>

namespace ibf {

constexpr int kTcThreads = 128;        // one MMA row per thread: M = 128
constexpr int kTcCols = 128;           // tensor-memory columns per CTA
constexpr int kTcK1 = 24, kTcK2 = 16;  // K extents of the two product sets
constexpr int kTcN = 32;               // outputs of both children, 16 apart
constexpr int kTcLBO = 128;            // bytes between K-adjacent 8x16B core matrices
constexpr int kTcB1Bytes = kTcN * kTcK1 * 4, kTcB2Bytes = kTcN * kTcK2 * 4;
// tensor-memory columns of one CTA: A rows (re, im), accumulators (re, im)
constexpr uint32_t kTcAre = 0, kTcAim = 32, kTcDre = 64, kTcDim = 96;
// bounded waits: polls of the MMA-completion barrier before giving up
constexpr int kTcMaxPolls = 1 << 22;

// B operands of one r in the byte layout the MMA reads (K-major, no swizzle:
// element (n, k) at (n/8) SBO + (k/4) LBO + (n%8) 16 + (k%4) 4 bytes)
struct TcOps {
    float b1[kTcN * kTcK1];
    float b2[kTcN * kTcK2];
};

// per-CTA state of the tensor-core levels
struct TcCtx {
    uint32_t tmem;        // tensor-memory base address (lane 0, first column)
    uint32_t mbar;        // shared address of the MMA-completion barrier
    uint32_t b1, b2;      // shared addresses of the B operands
    uint32_t phase;       // parity of the barrier's next completion
    int* status;          // global error word (1: a wait expired)
    bool abort;           // a wait expired: no further MMAs are issued
};

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// shared-memory matrix descriptor (no swizzle, version 1)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kTcLBO >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ULL << 46);
}

// instruction descriptor: D f32, A and B tf32, both K-major, M = 128, N = 32
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(kTcIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

// bounded wait for completion `phase` of the barrier; false if it expired
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase)
{
    for (int i = 0; i < kTcMaxPolls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};\n" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void tc_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Veltkamp split of a (re, im) pair: hi with 11 significant bits, lo = x - hi
__device__ __forceinline__ void tc_split(float2 x, float2& hi, float2& lo)
{
    const float2 c = __fmul2_rn(x, make_float2(8193.f, 8193.f));
    const float2 t = __ffma2_rn(x, make_float2(-1.f, -1.f), c);
    hi = __ffma2_rn(t, make_float2(-1.f, -1.f), c);
    lo = __ffma2_rn(hi, make_float2(-1.f, -1.f), x);
}

// CTA set-up: B operands into shared memory, barrier, tensor memory; ends
// with a barrier.  Called by all kTcThreads threads.
__device__ __forceinline__ void tc_setup(TcCtx& t, const TcOps& B, unsigned char* tail, int* status)
{
    float* b1 = reinterpret_cast<float*>(tail);
    float* b2 = b1 + kTcN * kTcK1;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(b2 + kTcN * kTcK2);
    uint32_t* taddr = reinterpret_cast<uint32_t*>(mbar + 1);
    for (int i = threadIdx.x; i < kTcN * kTcK1; i += blockDim.x) b1[i] = B.b1[i];
    for (int i = threadIdx.x; i < kTcN * kTcK2; i += blockDim.x) b2[i] = B.b2[i];
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc_smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc_smem_u32(taddr)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // B visible to the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    t.tmem = *taddr;
    t.mbar = tc_smem_u32(mbar);
    t.b1 = tc_smem_u32(b1);
    t.b2 = tc_smem_u32(b2);
    t.phase = 0;
    t.status = status;
    t.abort = false;
    // K padding of the A rows (columns 16..23 of each row block; 16..17 are
    // rewritten by every round, 18..23 stay zero)
    const uint32_t lane = (uint32_t)(threadIdx.x & ~31) << 16;
    const uint32_t z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    tc_st8(t.tmem + lane + kTcAre + 16, z);
    tc_st8(t.tmem + lane + kTcAim + 16, z);
    tc_wait_st();
}

// CTA tear-down: every tensor-memory access done, then free it.  After an
// expired wait, the MMAs still in flight get one more bounded wait first.
__device__ __forceinline__ void tc_teardown(TcCtx& t)
{
    if (t.abort) tc_wait(t.mbar, t.phase);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(t.tmem), "r"(kTcCols));
}

// One G-form butterfly level of the fused tile through the tensor cores: sm
// holds the Lambda tile ([pos][t][col], stride PS = r rt + 1), dl the staged
// tables of this level ([u], stride 4r, pair layout of tab_off for the level
// kind: G for the forward form, H for the adjoint).  Rounds of 128
// (unit, column) tasks; per round and input q: rows to tensor memory, five
// MMAs per component, products back, diagonals applied.  All threads take
// part in every round (the tensor-memory transfers are warp-collective).
template <int RP, bool ADJ, int RT>
__device__ __forceinline__ void tc_level_g(TcCtx& tc, int bit, int nunit, int rt_run, int ncol, float2* sm,
                                           const float2* dl)
{
    const int rt = RT ? RT : rt_run;
    const int PS = RP * rt + 1;
    constexpr int DS = 4 * RP;
    constexpr int KIND = ADJ ? 0 : 1;
    const uint32_t lane = (uint32_t)(threadIdx.x & ~31) << 16;
    const int ntask = nunit * rt;
    for (int r0 = 0; r0 < ntask; r0 += kTcThreads) {
        const int w = r0 + threadIdx.x;
        const int c = w % rt, u = w / rt;
        const bool on = w < ntask && c < ncol;
        const int p0 = ((u >> bit) << (bit + 1)) | (u & ((1 << bit) - 1));
        const int p1 = p0 | (1 << bit);
        const float2* du = dl + (size_t)u * DS;
        float2* o0 = sm + (size_t)p0 * PS + c;
        float2* o1 = sm + (size_t)p1 * PS + c;
        float2 y1[RP];   // output 1 until input 1 has been read; output 0 waits in place of input 0
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            // A rows of input q: [x_hi (RP) | x_lo (RP) | 0] for the real and imaginary parts
            {
                const float2* xp = q ? o1 : o0;
                uint32_t vr[16], vi[16], wr[8], wi[8];
#pragma unroll
                for (int j = 0; j < 16; ++j) vr[j] = vi[j] = 0u;
#pragma unroll
                for (int j = 0; j < 8; ++j) wr[j] = wi[j] = 0u;
#pragma unroll
                for (int s = 0; s < RP; ++s) {
                    const float2 x = on ? xp[s * rt] : make_float2(0.f, 0.f);
                    float2 hi, lo;
                    tc_split(x, hi, lo);
                    if (s < 16) {
                        vr[s] = __float_as_uint(hi.x);
                        vi[s] = __float_as_uint(hi.y);
                    } else {
                        wr[s - 16] = __float_as_uint(hi.x);
                        wi[s - 16] = __float_as_uint(hi.y);
                    }
                    if (RP + s < 16) {
                        vr[RP + s] = __float_as_uint(lo.x);
                        vi[RP + s] = __float_as_uint(lo.y);
                    } else {
                        wr[RP + s - 16] = __float_as_uint(lo.x);
                        wi[RP + s - 16] = __float_as_uint(lo.y);
                    }
                }
                tc_st16(tc.tmem + lane + kTcAre, vr);
                tc_st8(tc.tmem + lane + kTcAre + 16, wr);
                tc_st16(tc.tmem + lane + kTcAim, vi);
                tc_st8(tc.tmem + lane + kTcAim + 16, wi);
                tc_wait_st();
            }
            tc_fence_before();
            // every row stored, every earlier read of the accumulators done
            const bool abort = __syncthreads_or(tc.abort);
            tc_fence_after();
            tc.abort = abort;
            if (!abort) {
                if (threadIdx.x == 0) {
                    const uint32_t sbo1 = (kTcK1 / 4) * kTcLBO, sbo2 = (kTcK2 / 4) * kTcLBO;
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        const uint32_t A = tc.tmem + (part ? kTcAim : kTcAre);
                        const uint32_t D = tc.tmem + (part ? kTcDim : kTcDre);
#pragma unroll
                        for (int kk = 0; kk < kTcK1 / 8; ++kk)
                            tc_mma(D, A + kk * 8, tc_desc(tc.b1 + kk * 2 * kTcLBO, sbo1), kk > 0);
#pragma unroll
                        for (int kk = 0; kk < kTcK2 / 8; ++kk)
                            tc_mma(D, A + kk * 8, tc_desc(tc.b2 + kk * 2 * kTcLBO, sbo2), 1);
                    }
                    tc_commit(tc.mbar);
                }
                if (!tc_wait(tc.mbar, tc.phase)) {
                    tc.abort = true;
                    if (tc.status) atomicExch(tc.status, 1);
                } else {
                    tc.phase ^= 1;
                }
            }
            tc_fence_after();
            // products of child a at columns 16 a + t; out_a[t] += D_{a,q}[t] z_{q,a}[t]
            // (forward G); adjoint H: out_a[t] += conj(D_{q,a}[t]) z_{q,a}[t]
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                uint32_t zr[16], zi[16];
                tc_ld16(tc.tmem + lane + kTcDre + 16 * a, zr);
                tc_ld16(tc.tmem + lane + kTcDim + 16 * a, zi);
                tc_wait_ld();
                const int ac = ADJ ? (q * 2 + a) : (a * 2 + q);
                const float2* dA = du + tab_off<RP, KIND>(ac, 0);
                if (on) {
#pragma unroll
                    for (int t = 0; t < RP; ++t) {
                        const float2 z = make_float2(__uint_as_float(zr[t]), __uint_as_float(zi[t]));
                        if (a == 0) {
                            // input 0 is consumed: output 0 accumulates in its place
                            float2 y = q ? o0[t * rt] : make_float2(0.f, 0.f);
                            cmacx<ADJ>(y, dA[2 * t], z);
                            o0[t * rt] = y;
                        } else {
                            if (q == 0) y1[t] = make_float2(0.f, 0.f);
                            cmacx<ADJ>(y1[t], dA[2 * t], z);
                        }
                    }
                }
            }
        }
        if (on) {
#pragma unroll
            for (int t = 0; t < RP; ++t) o1[t * rt] = y1[t];
        }
    }
}

// B operands of the G form for the plan's T_c (host): B1 rows 0..RP-1 and
// RP..2RP-1 hold w_hi, B2 rows 0..RP-1 hold w_lo, with w = T_a[s][t] for
// output n = 16 a + t and input k = s (K-major, no swizzle)
inline void tc_build_ops(const double (*T0)[16], const double (*T1)[16], int RP, TcOps& B)
{
    memset(&B, 0, sizeof(B));
    auto at = [](float* base, int Ktot, int n, int k) -> float& {
        const int sbo = (Ktot / 4) * kTcLBO;
        const size_t byte = (size_t)(n / 8) * sbo + (size_t)(k / 4) * kTcLBO + (n % 8) * 16 + (k % 4) * 4;
        return base[byte / 4];
    };
    for (int a = 0; a < 2; ++a)
        for (int t = 0; t < RP; ++t)
            for (int s = 0; s < RP; ++s) {
                const double w = (a ? T1 : T0)[s][t];
                // round to the 11 significant bits of TF32 (ties away from zero), then the remainder
                float wf = (float)w;
                uint32_t bits;
                memcpy(&bits, &wf, 4);
                bits = (bits + 0x1000u) & 0xFFFFE000u;
                float hi;
                memcpy(&hi, &bits, 4);
                const float lo = (float)(w - (double)hi);
                const int n = 16 * a + t;
                at(B.b1, kTcK1, n, s) = hi;
                at(B.b1, kTcK1, n, RP + s) = hi;
                at(B.b2, kTcK2, n, s) = lo;
            }
}

}  // namespace ibf
