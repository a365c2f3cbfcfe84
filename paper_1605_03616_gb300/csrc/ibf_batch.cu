// Batched apply of many structured-form plans of uneven size, and the
// launch-shape autotuner.
//
// A batch binds, once, a list of plans with their input/output buffers and
// right-hand-side counts.  Each plan's apply is a short sequence of fused
// chunks (levels fused per launch); the batch runs chunk p of every plan in
// one launch of k_fused_batch per (level kind, tile width, fusion depth) (CTA
// ranges map to plans through a prefix sum), so the launch count depends on
// the shapes present, not on the number of plans, and ibf_batch_apply issues
// nothing but those launches: it can be captured in a CUDA graph.
#include <algorithm>
#include <vector>

#include "ibf_fused.cuh"

struct ibf_batch {
    int dtype = 0, r = 0, adjoint = 0, count = 0;
    std::vector<int> nrhs;
    struct Phase {
        ibf::FusedDesc* descs = nullptr;   // device
        int64_t* start = nullptr;          // device, n entries
        int n = 0;
        int64_t blocks = 0;
        size_t smem = 0;
        int threads = 0;
        int kind = 0, rt = 0;
    };
    std::vector<Phase> phases;
    // persistent single-launch form: descriptors in chunk-major order
    ibf::FusedDesc* p_descs = nullptr;
    int64_t* p_start = nullptr;
    int* p_dep = nullptr;
    int64_t* p_need = nullptr;
    int* p_done = nullptr;
    unsigned long long* p_next = nullptr;
    int* p_status = nullptr;
    int p_n = 0;
    int64_t p_total = 0;
    size_t p_smem = 0;
    long long p_max_spin = 1LL << 21;
    std::vector<int64_t> p_need_host;
    std::vector<int> p_plan_of, p_chunk_of;
    std::vector<ibf_plan*> plans;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    std::vector<void*> allocations;
};

namespace ibf {

// Persistent batched launch: CTAs take work items (one CTA-sized block of one
// descriptor) from an atomic counter in descriptor order.  Descriptors are
// ordered chunk-major, so every item a block waits for was handed out before
// it, to a CTA that is already running: the waits cannot deadlock.  A block of
// chunk c of a plan waits until all blocks of that plan's chunk c-1 have
// finished (dep/need), with a bounded spin; on expiry it raises *status and
// every CTA stops.  Inputs written earlier in the same launch are read with
// L1-bypassing loads.
struct PersistArgs {
    const FusedDesc* descs;
    const int64_t* start;      // first item of each descriptor (n entries)
    const int* dep;            // descriptor this one waits for, or -1
    const int64_t* need;       // blocks of dep that must be done
    int* done;                 // finished blocks per descriptor (zeroed per apply)
    unsigned long long* next;  // work counter (zeroed per apply)
    int* status;               // 0, or 1 after a wait expired
    int64_t total;
    int n;
    long long max_spin;
};

// Persistent form: 256 threads per CTA (fusion depth at most 4 with 32-column
// tiles), as many CTAs as fit on the device at once.
// items a CTA claims at a time: consecutive items mostly share a descriptor,
// so the lookup, publish and dependency check run once per run of items
constexpr int kPersistRun = 8;

template <typename Real>
struct PersistTraits {
    static constexpr int kThreads = 256;
    // FP32: 4 CTAs per SM (64 registers); the two level kinds are separate
    // functions (persist_item), so the kernel holds one kind's registers at a time
    static constexpr int kMinBlocks = sizeof(Real) == 4 ? 4 : 1;
};

// One work item of one level kind, not inlined into the persistent loop: the
// loop keeps only its own state live across the call.
template <typename Real, int RP, bool ADJ, int KIND>
__device__ __noinline__ void persist_item(const FusedDesc& d, int64_t blk, unsigned char* smraw)
{
    fused_body<Real, RP, ADJ, KIND, 32, true>(c_eo<Real, RP>, d, blk, smraw);
}

// Each CTA takes runs of kPersistRun consecutive items from the shared counter
// in order (the next run is claimed while the current one runs, hiding the
// atomic's latency).  An item
// of a descriptor with a dependency may start once every item of that
// dependency is done; a CTA checks this once per run of items of the same
// descriptor.  Finished items are published (fence, then one atomic add per
// run) whenever the CTA moves to another descriptor and when it exits, so a
// CTA never waits while it holds unpublished work.  Waits are bounded: after
// max_spin polls the CTA sets the sticky status and every waiting CTA gives up.
template <typename Real, int RP, bool ADJ>
__global__ void __launch_bounds__(PersistTraits<Real>::kThreads, PersistTraits<Real>::kMinBlocks)
    k_fused_persist(const __grid_constant__ PersistArgs A)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ long long s_item[2];
    __shared__ int s_stop;
    int cur = -1;                       // descriptor of the current run of items
    int64_t cur_lo = 0, cur_hi = 0;     // its item range
    int pending = 0;                    // thread 0: finished items of cur not yet published
    if (threadIdx.x == 0) s_item[0] = (long long)atomicAdd(A.next, (unsigned long long)kPersistRun);
    __syncthreads();
    bool stop = false;
    for (int it = 0; !stop; ++it) {
        const long long base = s_item[it & 1];
        if (base >= A.total) break;
        // claim the next run while this one runs
        if (threadIdx.x == 0) s_item[(it + 1) & 1] = (long long)atomicAdd(A.next, (unsigned long long)kPersistRun);
        const long long end = min(base + (long long)kPersistRun, (long long)A.total);
        for (long long item = base; item < end; ++item) {
            if (item < cur_lo || item >= cur_hi) {
                if (cur >= 0) {
                    __threadfence();   // this thread's outputs are visible device-wide ...
                    __syncthreads();   // ... for every thread of the block ...
                    if (threadIdx.x == 0 && pending) atomicAdd(A.done + cur, pending);   // ... then counted
                    pending = 0;
                }
                int lo = cur > 0 ? cur : 0, hi = A.n - 1;   // items only increase
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (A.start[mid] <= item)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                cur = lo;
                cur_lo = A.start[lo];
                cur_hi = lo + 1 < A.n ? A.start[lo + 1] : A.total;
                const int dep = A.dep[lo];
                if (dep >= 0) {
                    if (threadIdx.x == 0) {
                        long long spins = 0;
                        int ok = 1;
                        while (atomicAdd(A.done + dep, 0) < A.need[lo]) {
                            if (++spins > A.max_spin || *(volatile int*)A.status) {
                                ok = 0;
                                break;
                            }
                            __nanosleep(200);
                        }
                        if (!ok) atomicExch(A.status, 1);
                        __threadfence();
                        s_stop = !ok;
                    }
                    __syncthreads();
                    if (s_stop) {
                        stop = true;
                        break;
                    }
                }
            }
            const FusedDesc& d = A.descs[cur];
            const int64_t blk = item - cur_lo;
            // every descriptor of the persistent form uses 32-column tiles
            if (d.kind == 0)
                persist_item<Real, RP, ADJ, 0>(d, blk, smraw);
            else
                persist_item<Real, RP, ADJ, 1>(d, blk, smraw);
            if (threadIdx.x == 0) ++pending;
            __syncthreads();   // shared memory and the claimed items change hands
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && cur >= 0 && pending) atomicAdd(A.done + cur, pending);
}


static int balloc(ibf_batch* b, void** ptr, size_t bytes)
{
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return set_error(IBF_ERR_OOM, "batch: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    b->allocations.push_back(*ptr);
    return IBF_OK;
}

static void batch_free(ibf_batch* b)
{
    if (!b) return;
    for (void* a : b->allocations) cudaFree(a);
    delete b;
}

template <typename Real, int RP, bool ADJ, int KIND, int RT>
static void batch_one(const FusedConsts<Real, RP>& C, const ibf_batch::Phase& ph, cudaStream_t st)
{
    static bool done = false;
    if (!done) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncSetAttribute(k_fused_batch<Real, RP, ADJ, KIND, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin);
        done = true;
    }
    k_fused_batch<Real, RP, ADJ, KIND, RT><<<(unsigned)ph.blocks, ph.threads, ph.smem, st>>>(C, ph.descs, ph.start,
                                                                                            ph.n);
}

template <typename Real, int RP, bool ADJ>
static void batch_kind(const FusedConsts<Real, RP>& C, const ibf_batch::Phase& ph, cudaStream_t st)
{
    if (ph.kind == 0) {
        if (ph.rt == 32)
            batch_one<Real, RP, ADJ, 0, 32>(C, ph, st);
        else
            batch_one<Real, RP, ADJ, 0, 0>(C, ph, st);
    } else {
        if (ph.rt == 32)
            batch_one<Real, RP, ADJ, 1, 32>(C, ph, st);
        else
            batch_one<Real, RP, ADJ, 1, 0>(C, ph, st);
    }
}

template <typename Real, int RP>
static int batch_launch(const ibf_batch* b, cudaStream_t st)
{
    FusedConsts<Real, RP> C;   // kernel argument kept for the launch signature
    memset(&C, 0, sizeof(C));
    for (const auto& ph : b->phases) {
        if (b->adjoint)
            batch_kind<Real, RP, true>(C, ph, st);
        else
            batch_kind<Real, RP, false>(C, ph, st);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : cuda_error(e, "batch launch");
}

template <typename Real, int RP>
static int persist_launch(const ibf_batch* b, cudaStream_t st)
{
    static bool attr = false;
    static int nsm = 0;
    if (!attr) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        // the kernel has a few bytes of static shared memory: the dynamic
        // limit is the opt-in maximum minus those
        cudaFuncAttributes fa;
        cudaFuncGetAttributes(&fa, k_fused_persist<Real, RP, false>);
        cudaFuncSetAttribute(k_fused_persist<Real, RP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
        cudaFuncGetAttributes(&fa, k_fused_persist<Real, RP, true>);
        cudaFuncSetAttribute(k_fused_persist<Real, RP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
        attr = true;
    }
    // every CTA must be resident at once (items wait on other CTAs' items)
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_persist<Real, RP, false>,
                                                      PersistTraits<Real>::kThreads, b->p_smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return set_error(IBF_ERR_CUDA, "persistent batch: the CTA shape does not fit an SM");
    }
    const int grid = nsm * per_sm;
    PersistArgs A;
    A.descs = b->p_descs;
    A.start = b->p_start;
    A.dep = b->p_dep;
    A.need = b->p_need;
    A.done = b->p_done;
    A.next = b->p_next;
    A.status = b->p_status;
    A.total = b->p_total;
    A.n = b->p_n;
    A.max_spin = b->p_max_spin;
    cudaMemsetAsync(b->p_done, 0, sizeof(int) * b->p_n, st);
    cudaMemsetAsync(b->p_next, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(b->p_status, 0, sizeof(int), st);
    const unsigned g = (unsigned)std::min<int64_t>(grid, b->p_total);
    if (b->adjoint)
        k_fused_persist<Real, RP, true><<<g, PersistTraits<Real>::kThreads, b->p_smem, st>>>(A);
    else
        k_fused_persist<Real, RP, false><<<g, PersistTraits<Real>::kThreads, b->p_smem, st>>>(A);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : cuda_error(e, "persistent batch launch");
}

template <typename Real>
static int persist_dispatch(const ibf_batch* b, cudaStream_t st)
{
    switch (b->r) {
    case 5: return persist_launch<Real, 5>(b, st);
    case 7: return persist_launch<Real, 7>(b, st);
    case 9: return persist_launch<Real, 9>(b, st);
    case 11: return persist_launch<Real, 11>(b, st);
    default: return set_error(IBF_ERR_UNSUPPORTED, "batch: unsupported r");
    }
}

template <typename Real>
static int batch_dispatch(const ibf_batch* b, cudaStream_t st)
{
    switch (b->r) {
    case 5: return batch_launch<Real, 5>(b, st);
    case 7: return batch_launch<Real, 7>(b, st);
    case 9: return batch_launch<Real, 9>(b, st);
    case 11: return batch_launch<Real, 11>(b, st);
    default: return set_error(IBF_ERR_UNSUPPORTED, "batch: unsupported r");
    }
}

}  // namespace ibf

using namespace ibf;

extern "C" int ibf_batch_create(ibf_plan* const* plans, int count, const int* nrhs, const void* const* in,
                                void* const* out, int adjoint, ibf_batch** outb)
{
    if (!outb) return set_error(IBF_ERR_INVALID, "batch: out is NULL");
    *outb = nullptr;
    if (!plans || !nrhs || !in || !out || count < 1) return set_error(IBF_ERR_INVALID, "batch: bad arguments");
    const ibf_plan* p0 = plans[0];
    if (!p0) return set_error(IBF_ERR_INVALID, "batch: NULL plan");
    for (int b = 0; b < count; ++b) {
        const ibf_plan* p = plans[b];
        if (!p) return set_error(IBF_ERR_INVALID, "batch: NULL plan");
        if (p->form != IBF_FORM_STRUCTURED) return set_error(IBF_ERR_UNSUPPORTED, "batch: plans must be structured");
        if (p->dtype != p0->dtype || p->r != p0->r)
            return set_error(IBF_ERR_INVALID, "batch: plans must share dtype and r");
        if (nrhs[b] < 1) return set_error(IBF_ERR_INVALID, "batch: nrhs must be >= 1");
        if (!in[b] || !out[b]) return set_error(IBF_ERR_INVALID, "batch: NULL vector pointer");
    }
    const size_t esz = p0->dtype == IBF_C128 ? sizeof(double2) : sizeof(float2);
    ibf_batch* B = new ibf_batch();
    B->dtype = p0->dtype;
    B->r = p0->r;
    B->adjoint = adjoint ? 1 : 0;
    B->count = count;
    B->plans.assign(plans, plans + count);
    B->nrhs.assign(nrhs, nrhs + count);

    // per-plan schedules and workspace offsets
    std::vector<std::vector<Chunk>> sched(count);
    std::vector<int> rt(count);
    std::vector<size_t> wsoff(count);
    size_t ws = 0;
    int nphase = 0;
    for (int b = 0; b < count; ++b) {
        const ibf_plan* p = plans[b];
        rt[b] = std::min(32, pow2ceil(nrhs[b]));
        if (p->user_rtile) rt[b] = std::min(rt[b], p->rtile);
        int kmax = p->user_kfuse ? p->kfuse : fused_kmax(rt[b], p->r, esz);
        sched[b] = fused_schedule(p->L, p->h, std::max(1, std::min(kmax, kMaxFuse)));
        nphase = std::max(nphase, (int)sched[b].size());
        wsoff[b] = ws;
        ws += ((2 * esz * (size_t)p->N * p->r * nrhs[b]) + 255) / 256 * 256;
    }
    int rc = balloc(B, &B->ws, ws);
    if (rc) {
        batch_free(B);
        return rc;
    }
    B->ws_bytes = ws;

    // one launch per (chunk index, level kind, tile width, fusion depth): every
    // CTA of a launch has exactly the shape its chunk needs, (2^k / 2) * rt
    // threads and the shared memory of depth k
    const int cap = p0->dtype == IBF_C128 ? FusedTraits<double>::kThreads : FusedTraits<float>::kThreads;
    for (int ph = 0; ph < nphase; ++ph) {
        for (int kc = 0; kc < 2; ++kc)
        for (int rtc = 1; rtc <= 32; rtc *= 2)
        for (int kq = 1; kq <= kMaxFuse; ++kq) {
            std::vector<FusedDesc> descs;
            std::vector<int64_t> start;
            int64_t blocks = 0;
            size_t smem = 0;
            int threads = 32;
            for (int b = 0; b < count; ++b) {
                const int nch = (int)sched[b].size();
                if (ph >= nch || rt[b] != rtc) continue;
                const ibf_plan* p = plans[b];
                const Chunk ch = B->adjoint ? sched[b][nch - 1 - ph] : sched[b][ph];
                if (ch.kind != kc || ch.hi - ch.lo != kq) continue;
                FusedDesc d;
                memset(&d, 0, sizeof(d));
                d.k = ch.hi - ch.lo;
                d.l0 = ch.lo;
                d.kind = ch.kind;
                for (int s = 1; s <= d.k; ++s) d.D[s - 1] = p->stab[ch.lo + s];
                if (!B->adjoint) {
                    d.pro = ch.lo == 0 ? PRO_V : PRO_LAMBDA;
                    d.epi = ch.hi == p->L ? EPI_U : (ch.hi == p->h ? EPI_SWITCH : EPI_LAMBDA);
                } else {
                    d.pro = ch.hi == p->L ? PRO_UADJ : PRO_LAMBDA;
                    d.epi = ch.lo == 0 ? EPI_VADJ : (ch.lo == p->h ? EPI_SWITCH : EPI_LAMBDA);
                }
                char* base = (char*)B->ws + wsoff[b];
                const size_t half = esz * (size_t)p->N * p->r * nrhs[b];
                d.in = base + (ph & 1) * half;
                d.out = base + ((ph & 1) ^ 1) * half;
                d.vin = in[b];
                d.vout = out[b];
                d.Vs = p->sV;
                d.Us = p->sU;
                d.Ms = p->sM;
                d.perm = p->d_perm;
                d.off = p->d_off;
                d.N = p->N;
                d.L = p->L;
                d.nc = nrhs[b];
                d.rt = rt[b];
                descs.push_back(d);
                start.push_back(blocks);
                const int64_t ntile = (nrhs[b] + rt[b] - 1) / rt[b];
                blocks += (1LL << (p->L - d.k)) * ntile;
                smem = std::max(smem, fused_smem_bytes(d.k, rt[b], p->r, esz, d.pro));
                threads = std::max(threads, std::min(cap, (1 << (d.k - 1)) * rt[b]));
            }
            if (descs.empty()) continue;
            ibf_batch::Phase P;
            P.n = (int)descs.size();
            P.blocks = blocks;
            P.smem = smem;
            P.threads = (threads + 31) / 32 * 32;
            P.kind = kc;
            P.rt = rtc;
            if ((rc = balloc(B, (void**)&P.descs, sizeof(FusedDesc) * descs.size())) ||
                (rc = balloc(B, (void**)&P.start, sizeof(int64_t) * start.size()))) {
                batch_free(B);
                return rc;
            }
            cudaMemcpy(P.descs, descs.data(), sizeof(FusedDesc) * descs.size(), cudaMemcpyHostToDevice);
            cudaMemcpy(P.start, start.data(), sizeof(int64_t) * start.size(), cudaMemcpyHostToDevice);
            B->phases.push_back(P);
        }
    }
    // persistent form: the same chunks, chunk-major, each waiting for its plan's previous chunk
    {
        std::vector<FusedDesc> descs;
        std::vector<int64_t> start, need;
        std::vector<int> dep;
        std::vector<int> last(count, -1);
        std::vector<int64_t> last_blocks(count, 0);
        int64_t total = 0;
        size_t smem = 0;
        // one CTA shape for the whole launch: 32-column tiles and a fusion
        // depth whose butterfly steps fill the CTA (2^(k-1) x 32 <= threads)
        std::vector<std::vector<Chunk>> psched(count);
        int pphase = 0;
        const int kcta = 4;   // 2^(4-1) x 32 = 256 threads, the persistent CTA
        for (int b = 0; b < count; ++b) {
            const ibf_plan* p = plans[b];
            const int kfit = std::min(kcta, fused_kmax(32, p->r, esz));
            const int kmax = p->user_kfuse ? std::min(p->kfuse, kfit) : kfit;
            psched[b] = fused_schedule(p->L, p->h, std::max(1, kmax));
            pphase = std::max(pphase, (int)psched[b].size());
        }
        for (int ph = 0; ph < pphase; ++ph)
            for (int b = 0; b < count; ++b) {
                const int nch = (int)psched[b].size();
                if (ph >= nch) continue;
                const ibf_plan* p = plans[b];
                const Chunk ch = B->adjoint ? psched[b][nch - 1 - ph] : psched[b][ph];
                FusedDesc d;
                memset(&d, 0, sizeof(d));
                d.k = ch.hi - ch.lo;
                d.l0 = ch.lo;
                d.kind = ch.kind;
                for (int s = 1; s <= d.k; ++s) d.D[s - 1] = p->stab[ch.lo + s];
                if (!B->adjoint) {
                    d.pro = ch.lo == 0 ? PRO_V : PRO_LAMBDA;
                    d.epi = ch.hi == p->L ? EPI_U : (ch.hi == p->h ? EPI_SWITCH : EPI_LAMBDA);
                } else {
                    d.pro = ch.hi == p->L ? PRO_UADJ : PRO_LAMBDA;
                    d.epi = ch.lo == 0 ? EPI_VADJ : (ch.lo == p->h ? EPI_SWITCH : EPI_LAMBDA);
                }
                char* base = (char*)B->ws + wsoff[b];
                const size_t half = esz * (size_t)p->N * p->r * nrhs[b];
                d.in = base + (ph & 1) * half;
                d.out = base + ((ph & 1) ^ 1) * half;
                d.vin = in[b];
                d.vout = out[b];
                d.Vs = p->sV;
                d.Us = p->sU;
                d.Ms = p->sM;
                d.perm = p->d_perm;
                d.off = p->d_off;
                d.N = p->N;
                d.L = p->L;
                d.nc = nrhs[b];
                d.rt = 32;   // one CTA shape for the whole launch
                const int64_t blocks = (1LL << (p->L - d.k)) * ((nrhs[b] + 31) / 32);
                dep.push_back(last[b]);
                need.push_back(last[b] >= 0 ? last_blocks[b] : 0);
                B->p_plan_of.push_back(b);
                B->p_chunk_of.push_back(ph);
                last[b] = (int)descs.size();
                last_blocks[b] = blocks;
                descs.push_back(d);
                start.push_back(total);
                total += blocks;
                smem = std::max(smem, fused_smem_bytes(d.k, 32, p->r, esz, d.pro));
            }
        B->p_n = (int)descs.size();
        B->p_total = total;
        B->p_smem = smem;
        B->p_need_host = need;
        if ((rc = balloc(B, (void**)&B->p_descs, sizeof(FusedDesc) * descs.size())) ||
            (rc = balloc(B, (void**)&B->p_start, sizeof(int64_t) * start.size())) ||
            (rc = balloc(B, (void**)&B->p_dep, sizeof(int) * dep.size())) ||
            (rc = balloc(B, (void**)&B->p_need, sizeof(int64_t) * need.size())) ||
            (rc = balloc(B, (void**)&B->p_done, sizeof(int) * descs.size())) ||
            (rc = balloc(B, (void**)&B->p_next, sizeof(unsigned long long))) ||
            (rc = balloc(B, (void**)&B->p_status, sizeof(int)))) {
            batch_free(B);
            return rc;
        }
        cudaMemcpy(B->p_descs, descs.data(), sizeof(FusedDesc) * descs.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(B->p_start, start.data(), sizeof(int64_t) * start.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(B->p_dep, dep.data(), sizeof(int) * dep.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(B->p_need, need.data(), sizeof(int64_t) * need.size(), cudaMemcpyHostToDevice);
        cudaMemset(B->p_status, 0, sizeof(int));
    }
    rc = p0->dtype == IBF_C128 ? fused_upload_consts<double>(p0) : fused_upload_consts<float>(p0);
    if (rc) {
        batch_free(B);
        return rc;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        batch_free(B);
        return cuda_error(e, "batch set-up");
    }
    *outb = B;
    return IBF_OK;
}

extern "C" int ibf_batch_apply(const ibf_batch* b, ibf_stream_t stream)
{
    if (!b) return set_error(IBF_ERR_INVALID, "batch is NULL");
    if (b->dtype == IBF_C128) return batch_dispatch<double>(b, (cudaStream_t)stream);
    return batch_dispatch<float>(b, (cudaStream_t)stream);
}

extern "C" int ibf_batch_apply_persistent(const ibf_batch* b, ibf_stream_t stream)
{
    if (!b) return set_error(IBF_ERR_INVALID, "batch is NULL");
    if (b->p_total <= 0) return IBF_OK;
    if (b->dtype == IBF_C128) return persist_dispatch<double>(b, (cudaStream_t)stream);
    return persist_dispatch<float>(b, (cudaStream_t)stream);
}

extern "C" int ibf_batch_status(const ibf_batch* b)
{
    if (!b) return set_error(IBF_ERR_INVALID, "batch is NULL");
    int st = 0;
    cudaError_t e = cudaMemcpy(&st, b->p_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "batch status");
    if (st) {
        for (ibf_plan* p : b->plans) plan_note(p, IBF_ERR_TIMEOUT);
        return set_error(IBF_ERR_TIMEOUT, "persistent batch: a dependency wait expired");
    }
    return IBF_OK;
}

extern "C" int ibf_batch_set_wait_limit(ibf_batch* b, long long spins)
{
    if (!b || spins < 1) return set_error(IBF_ERR_INVALID, "bad batch or spin limit");
    b->p_max_spin = spins;
    return IBF_OK;
}

extern "C" int ibf_batch_test_withhold(ibf_batch* b, int plan, int withhold)
{
    if (!b || plan < 0 || plan >= b->count) return set_error(IBF_ERR_INVALID, "bad batch or plan index");
    for (int d = 0; d < b->p_n; ++d) {
        if (b->p_plan_of[d] != plan || b->p_chunk_of[d] != 1) continue;
        const int64_t v = withhold ? ((int64_t)1 << 40) : b->p_need_host[d];
        cudaError_t e = cudaMemcpy(b->p_need + d, &v, sizeof(int64_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_error(e, "batch test hook");
        return IBF_OK;
    }
    return set_error(IBF_ERR_INVALID, "plan has a single chunk: nothing to withhold");
}

extern "C" int ibf_batch_query(const ibf_batch* b, int what, int64_t* v)
{
    if (!b || !v) return set_error(IBF_ERR_INVALID, "NULL argument");
    switch (what) {
    case IBF_BQ_LAUNCHES: *v = (int64_t)b->phases.size(); break;
    case IBF_BQ_WORKSPACE_BYTES: *v = (int64_t)b->ws_bytes; break;
    case IBF_BQ_COUNT: *v = b->count; break;
    case IBF_BQ_PERSIST_ITEMS: *v = b->p_total; break;
    default: return set_error(IBF_ERR_INVALID, "unknown batch query");
    }
    return IBF_OK;
}

extern "C" int ibf_batch_destroy(ibf_batch* b)
{
    if (!b) return IBF_OK;
    cudaDeviceSynchronize();
    batch_free(b);
    return IBF_OK;
}

// Launch-shape autotuner: time the forward apply of this plan for each
// candidate (levels per launch, rhs tile) on scratch buffers and keep the
// fastest.  Candidates: tiles 8, 16, 32 (not above the next power of two of
// nrhs) and every fusion depth from 2 to the largest that keeps two CTAs per
// SM.
extern "C" int ibf_plan_autotune(ibf_plan* p, int nrhs, ibf_stream_t stream, int* best_k, int* best_rt,
                                 float* best_ms)
{
    if (!p || nrhs < 1) return set_error(IBF_ERR_INVALID, "autotune: bad arguments");
    if (p->form != IBF_FORM_STRUCTURED) return set_error(IBF_ERR_UNSUPPORTED, "autotune: structured plans only");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t esz = p->dtype == IBF_C128 ? sizeof(double2) : sizeof(float2);
    const size_t bytes = esz * (size_t)p->N * nrhs;
    void *g = nullptr, *u = nullptr;
    if (cudaMalloc(&g, bytes) != cudaSuccess || cudaMalloc(&u, bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(g);
        return set_error(IBF_ERR_OOM, "autotune: scratch allocation failed");
    }
    cudaMemsetAsync(g, 0, bytes, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool uk = p->user_kfuse, ur = p->user_rtile;
    const int ok = p->kfuse, orr = p->rtile;
    float best = 1e30f;
    int bk = ok, br = orr, rc = IBF_OK;
    const int rmax = std::min(32, pow2ceil(std::min(nrhs, p->max_nrhs)));
    for (int rt = 8; rt <= 32; rt *= 2) {
        if (rt > rmax && rt != 8) break;
        const int rtc = std::min(rt, rmax);
        for (int k = 2; k <= fused_kmax(rtc, p->r, esz); ++k) {
            p->user_kfuse = p->user_rtile = true;
            p->kfuse = k;
            p->rtile = rtc;
            rc = fused_apply(p, g, u, nrhs, false, st);   // warm-up
            if (rc) break;
            cudaEventRecord(e0, st);
            for (int it = 0; it < 3; ++it) fused_apply(p, g, u, nrhs, false, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3;
            if (ms < best) {
                best = ms;
                bk = k;
                br = rtc;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(g);
    cudaFree(u);
    if (rc) {
        p->user_kfuse = uk;
        p->user_rtile = ur;
        p->kfuse = ok;
        p->rtile = orr;
        return rc;
    }
    p->user_kfuse = p->user_rtile = true;
    p->kfuse = bk;
    p->rtile = br;
    if (best_k) *best_k = bk;
    if (best_rt) *best_rt = br;
    if (best_ms) *best_ms = best;
    return IBF_OK;
}
