// prec_f32.cu -- kernel instantiations for SMRT_PREC_F32 storage.
#include "kernels.cuh"

namespace smrt {
const KernelTable &kernels_f32()
{
    static const KernelTable t = make_table<SMRT_PREC_F32>();
    return t;
}
} // namespace smrt
