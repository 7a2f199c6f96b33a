// tds_fam_f32c.cu -- the FP32 with FP64 closure rows (TrNative<float, W, true>: closed lines with a
// high end gain) instantiations of the resident kernels of tds_resident.cuh, in a translation unit
// of their own so that the families compile in parallel.
#include "tds_resident.cuh"

namespace tds {
TDS_FAMILY_DEFINE_NATIVE(f32c, FamF32c)
} // namespace tds
