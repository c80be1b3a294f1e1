// placeholder, replaced by the batched persistent kernel
#include "kg_internal.h"
extern "C" {
kg_status kg_batch_create(kg_batch** out, kg_problem* const* probs, int count, const kg_options* opt, kg_stream s) { return KG_ERR_UNSUPPORTED; }
kg_status kg_grad_batched(kg_batch* b, const void* const* x, void* const* f, void* const* gx, kg_stream s) { return KG_ERR_UNSUPPORTED; }
kg_status kg_grad_batched_loop(kg_batch* b, const void* const* x, void* const* f, void* const* gx, kg_stream s) { return KG_ERR_UNSUPPORTED; }
kg_status kg_batch_sync(kg_batch* b) { return KG_ERR_UNSUPPORTED; }
void kg_batch_destroy(kg_batch* b) {}
}
