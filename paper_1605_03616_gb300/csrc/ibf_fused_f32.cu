// FP32 instantiation of the structured fused apply, and the host-side
// dispatch shared by both precisions.
#include "ibf_fused.cuh"

namespace ibf {

int fused_apply_f64(ibf_plan* p, const void* vin, void* vout, int nrhs, bool adj, cudaStream_t st);
int fused_prepare_f64(const ibf_plan* p);

int fused_apply(ibf_plan* p, const void* vin, void* vout, int nrhs, bool adj, cudaStream_t st)
{
    if (p->dtype == IBF_C128) return fused_apply_f64(p, vin, vout, nrhs, adj, st);
    return fused_apply_t<float>(p, vin, vout, nrhs, adj, st);
}

bool fused_supports_r(int r) { return r == 5 || r == 7 || r == 9 || r == 11; }

void fused_choose_shape(ibf_plan* p)
{
    // weights into constant memory now, outside any stream capture
    if (p->dtype == IBF_C128)
        fused_prepare_f64(p);
    else
        fused_upload_consts<float>(p);
    const size_t esz = p->dtype == IBF_C128 ? sizeof(double2) : sizeof(float2);
    if (!p->user_rtile) p->rtile = std::min(32, pow2ceil(p->max_nrhs));
    if (!p->user_kfuse) p->kfuse = fused_kmax(p->rtile, p->r, esz);
}

int fused_launches(const ibf_plan* p) { return (int)fused_schedule(p->L, p->h, p->kfuse).size(); }

}  // namespace ibf
