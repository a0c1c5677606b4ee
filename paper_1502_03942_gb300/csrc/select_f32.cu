// select_f32.cu — the selection kernels of topk_select instantiated for
// f32 keys (both orders), in a translation unit of their own so that the
// key types compile in parallel.
#include "select_impl.cuh"

namespace topk {
TOPK_SELECT_TEMPLATES(, DT_F32)
} // namespace topk
