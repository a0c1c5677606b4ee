// select_u64.cu — the selection kernels of topk_select instantiated for
// u64 keys (both orders), in a translation unit of their own so that the
// key types compile in parallel.
#include "select_impl.cuh"

namespace topk {
TOPK_SELECT_TEMPLATES(, DT_U64)
} // namespace topk
