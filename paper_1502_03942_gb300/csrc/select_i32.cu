// select_i32.cu — the selection kernels of topk_select instantiated for
// i32 keys (both orders), in a translation unit of their own so that the
// key types compile in parallel.
#include "select_impl.cuh"

namespace topk {
TOPK_SELECT_TEMPLATES(, DT_I32)
} // namespace topk
