// ibf_apply_static_scratch: the structured-form apply with its scratch in a
// fixed, library-owned device array instead of the plan's workspace.
//
// Why: some callers may not allocate device memory once their plans exist --
// for example a plug-in inside a host application that owns the device heap
// and forbids further cudaMalloc calls, or a server whose memory budget was
// fixed when the plans were built.  Such a caller can create its plans with
// max_nrhs = 1 (the smallest workspace a plan owns) and still apply many
// right-hand sides per launch through this entry point, which allocates
// nothing: its two Lambda buffers live in the static array below.
//
// The array is a file-scope __device__ variable of this translation unit's
// module.  The module is loaded on a device (and the array committed there)
// when its address is first looked up; creating a 1D structured plan does
// that on the plan's device (static_scratch_prepare), so the memory is taken
// while the caller may still allocate, and stays taken until the process
// exits.  Host code must not pass the symbol itself to a kernel (on the host
// it names a stand-in, not device memory); the device address comes from
// cudaGetSymbolAddress, once per device, and is cached.
#include <mutex>

#include "ibf_fused.cuh"

namespace ibf {

// 256 MiB: two Lambda buffers of 128 MiB each.
constexpr size_t kStaticScratchBytes = size_t(256) << 20;
constexpr size_t kStaticHalf = kStaticScratchBytes / 2;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_addr[64] = {nullptr};

// This file's copy of the transfer weights for the plan's (precision, r).
static int static_upload_consts(const ibf_plan* p)
{
    const bool f64 = p->dtype == IBF_C128;
    switch (p->r) {
    case 5: return f64 ? fused_upload_consts_t<double, 5>(p) : fused_upload_consts_t<float, 5>(p);
    case 7: return f64 ? fused_upload_consts_t<double, 7>(p) : fused_upload_consts_t<float, 7>(p);
    case 9: return f64 ? fused_upload_consts_t<double, 9>(p) : fused_upload_consts_t<float, 9>(p);
    case 11: return f64 ? fused_upload_consts_t<double, 11>(p) : fused_upload_consts_t<float, 11>(p);
    default: return set_error(IBF_ERR_UNSUPPORTED, "structured form: unsupported r");
    }
}

// Set-up for the current device, under g_static_mu: the device address of
// g_static_scratch (the lookup loads this module and commits the array on
// the device) and the weights for the plan's (precision, r).  Only the
// first call per device and per (precision, r) makes CUDA calls that are not
// allowed during stream capture (module load, a synchronous symbol copy).
static int static_prepare_current(const ibf_plan* p, void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(IBF_ERR_UNSUPPORTED, "device index >= 64");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
        g_static_addr[dev] = ptr;
    }
    const int rc = static_upload_consts(p);
    if (rc) return rc;
    if (out) *out = g_static_addr[dev];
    return IBF_OK;
}

// Called when a 1D structured plan is created, on its device.
int static_scratch_prepare(const ibf_plan* p) { return static_prepare_current(p, nullptr); }

// The fused forward schedule of fused_run with caller-chosen Lambda buffers.
template <typename Real, int RP>
static int static_run(const ibf_plan* p, const void* vin, void* vout, int nrhs, cudaStream_t st, void* buf0,
                      void* buf1, int max_cols)
{
    typedef typename CT<Real>::T cx;
    FusedParams<Real, RP> P;
    memset(&P, 0, sizeof(P));
    P.d.Vs = p->sV;
    P.d.Us = p->sU;
    P.d.Ms = p->sM;
    P.d.perm = p->d_perm;
    P.d.off = p->d_off;
    P.d.N = p->N;
    P.d.L = p->L;
    const int64_t N = p->N;
    for (int c0 = 0; c0 < nrhs; c0 += max_cols) {
        const int nc = std::min(max_cols, nrhs - c0);
        const int rt = std::min(32, pow2ceil(nc));
        const int kmax = fused_kmax(rt, RP, sizeof(cx));
        std::vector<Chunk> sched = fused_schedule(p->L, p->h, kmax);
        P.d.nc = nc;
        P.d.rt = rt;
        P.d.vin = (const cx*)vin + N * c0;
        P.d.vout = (cx*)vout + N * c0;
        void* bufs[2] = {buf0, buf1};
        int cur = 0;
        for (const Chunk& ch : sched) {
            P.d.l0 = ch.lo;
            P.d.kind = ch.kind;
            P.d.k = ch.hi - ch.lo;
            for (int s = 1; s <= P.d.k; ++s) P.d.D[s - 1] = p->stab[ch.lo + s];
            for (int s = P.d.k; s < kMaxFuse; ++s) P.d.D[s] = nullptr;
            P.d.pro = ch.lo == 0 ? PRO_V : PRO_LAMBDA;
            P.d.epi = ch.hi == p->L ? EPI_U : (ch.hi == p->h ? EPI_SWITCH : EPI_LAMBDA);
            P.d.in = bufs[cur];
            P.d.out = bufs[cur ^ 1];
            const int64_t ngroups = 1LL << (p->L - P.d.k);
            if (ch.kind == 0)
                launch_one<Real, RP, false, 0>(P, ngroups, st);
            else
                launch_one<Real, RP, false, 1>(P, ngroups, st);
            cur ^= 1;
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : cuda_error(e, "static-scratch apply launch");
}

template <typename Real>
static int static_dispatch(const ibf_plan* p, const void* g, void* u, int nrhs, cudaStream_t st, void* b0, void* b1,
                           int max_cols)
{
    switch (p->r) {
    case 5: return static_run<Real, 5>(p, g, u, nrhs, st, b0, b1, max_cols);
    case 7: return static_run<Real, 7>(p, g, u, nrhs, st, b0, b1, max_cols);
    case 9: return static_run<Real, 9>(p, g, u, nrhs, st, b0, b1, max_cols);
    case 11: return static_run<Real, 11>(p, g, u, nrhs, st, b0, b1, max_cols);
    default: return set_error(IBF_ERR_UNSUPPORTED, "structured form: unsupported r");
    }
}

}  // namespace ibf

using namespace ibf;

extern "C" int ibf_apply_static_scratch(const ibf_plan* p, const void* g, void* u, int nrhs, ibf_stream_t stream)
{
    if (!p) return set_error(IBF_ERR_INVALID, "plan is NULL");
    if (!g || !u) return set_error(IBF_ERR_INVALID, "NULL vector pointer");
    if (nrhs < 1) return set_error(IBF_ERR_INVALID, "nrhs must be >= 1");
    if (p->d != 1) return set_error(IBF_ERR_UNSUPPORTED, "static-scratch apply needs a 1D plan");
    if (p->form != IBF_FORM_STRUCTURED)
        return set_error(IBF_ERR_UNSUPPORTED, "static-scratch apply needs a structured-form plan");
    if (!fused_supports_r(p->r)) return set_error(IBF_ERR_UNSUPPORTED, "structured form: unsupported r");
    const size_t esz = p->dtype == IBF_C128 ? sizeof(double2) : sizeof(float2);
    if (((uintptr_t)g % esz) || ((uintptr_t)u % esz)) return set_error(IBF_ERR_INVALID, "misaligned vector pointer");
    const size_t bytes = esz * (size_t)p->N * nrhs;
    const char* cg = (const char*)g;
    const char* cu = (const char*)u;
    if (cg < cu + bytes && cu < cg + bytes) return set_error(IBF_ERR_INVALID, "input and output overlap");
    const size_t col_bytes = esz * (size_t)p->N * p->r;   // one Lambda column
    if (col_bytes > kStaticHalf)
        return set_error(IBF_ERR_INVALID, "N*r*element size = " + std::to_string(col_bytes) +
                                              " bytes exceeds the static scratch limit of " +
                                              std::to_string(kStaticHalf) + " bytes per Lambda buffer");
    void* base = nullptr;
    int rc = static_prepare_current(p, &base);
    if (rc) return plan_note(p, rc);
    const int max_cols = (int)std::min<size_t>(kStaticHalf / col_bytes, 1 << 20);
    void* b0 = base;
    void* b1 = (char*)base + kStaticHalf;
    if (p->dtype == IBF_C128)
        return plan_note(p, static_dispatch<double>(p, g, u, nrhs, (cudaStream_t)stream, b0, b1, max_cols));
    return plan_note(p, static_dispatch<float>(p, g, u, nrhs, (cudaStream_t)stream, b0, b1, max_cols));
}
