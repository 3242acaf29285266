// stubs.cu -- entry points whose kernels are not built yet report UNSUPPORTED.
#include "system.cuh"
using namespace sp;
#define STUB(name, ...) sptrsv_status name(__VA_ARGS__) { set_error(#name ": not available in this build"); return SPTRSV_ERR_UNSUPPORTED; }
namespace sp {
sptrsv_status learned_rewrite(const sptrsv_csr*, const sptrsv_levels*, const sptrsv_strategy*, sptrsv_system**,
                              cudaStream_t) {
    set_error("learned rewrite: not available in this build");
    return SPTRSV_ERR_UNSUPPORTED;
}
}  // namespace sp
extern "C" {
STUB(sptrsv_batch_create, const sptrsv_system* const*, const int32_t*, int32_t, sptrsv_batch**, sptrsv_stream_t)
STUB(sptrsv_batch_solve, sptrsv_batch*, const void* const*, void* const*, sptrsv_stream_t)
STUB(sptrsv_batch_info_get, const sptrsv_batch*, sptrsv_batch_info*)
void sptrsv_batch_destroy(sptrsv_batch*) {}
STUB(sptrsv_picker_create, uint64_t, sptrsv_picker**)
void sptrsv_picker_destroy(sptrsv_picker*) {}
STUB(sptrsv_picker_get_params, const sptrsv_picker*, float*)
STUB(sptrsv_picker_set_params, sptrsv_picker*, const float*)
STUB(sptrsv_picker_set_norm, sptrsv_picker*, const float*, const float*, float)
STUB(sptrsv_picker_save, const sptrsv_picker*, const char*)
STUB(sptrsv_picker_load, sptrsv_picker*, const char*)
STUB(sptrsv_picker_features, const sptrsv_csr*, const sptrsv_levels*, const int32_t*, int32_t, float*, sptrsv_stream_t)
STUB(sptrsv_picker_infer, const sptrsv_picker*, const float*, int64_t, float*, int32_t, sptrsv_stream_t)
STUB(sptrsv_picker_grad, const sptrsv_picker*, const float*, const float*, int64_t, int32_t, float*, float*, sptrsv_stream_t)
STUB(sptrsv_picker_train_step, sptrsv_picker*, const float*, const float*, int64_t, float, float*, sptrsv_stream_t)
}
