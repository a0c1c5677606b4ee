// select_bf16.cu — the selection kernels of topk_select instantiated for
// bf16 keys (both orders), in a translation unit of their own so that the
// key types compile in parallel.
#include "select_impl.cuh"

namespace topk {
TOPK_SELECT_TEMPLATES(, DT_BF16)
} // namespace topk
