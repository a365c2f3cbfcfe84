// FP64 instantiation of the structured fused apply.
#include "ibf_fused.cuh"

namespace ibf {

int fused_apply_f64(ibf_plan* p, const void* vin, void* vout, int nrhs, bool adj, cudaStream_t st)
{
    return fused_apply_t<double>(p, vin, vout, nrhs, adj, st);
}

int fused_prepare_f64(const ibf_plan* p) { return fused_upload_consts<double>(p); }

}  // namespace ibf
