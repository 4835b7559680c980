// prec_bf16.cu -- kernel instantiations for SMRT_PREC_BF16 storage.
#include "kernels.cuh"

namespace smrt {
const KernelTable &kernels_bf16()
{
    static const KernelTable t = make_table<SMRT_PREC_BF16>();
    return t;
}
} // namespace smrt
