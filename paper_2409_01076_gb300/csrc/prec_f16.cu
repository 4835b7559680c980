// prec_f16.cu -- kernel instantiations for SMRT_PREC_F16 storage.
#include "kernels.cuh"

namespace smrt {
const KernelTable &kernels_f16()
{
    static const KernelTable t = make_table<SMRT_PREC_F16>();
    return t;
}
} // namespace smrt
