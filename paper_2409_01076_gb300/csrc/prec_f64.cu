// prec_f64.cu -- kernel instantiations for SMRT_PREC_F64 storage.
#include "kernels.cuh"

namespace smrt {
const KernelTable &kernels_f64()
{
    static const KernelTable t = make_table<SMRT_PREC_F64>();
    return t;
}
} // namespace smrt
