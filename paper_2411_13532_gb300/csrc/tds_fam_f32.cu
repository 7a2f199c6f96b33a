// tds_fam_f32.cu -- the FP32 (TrNative<float, W>) instantiations of the resident kernels of
// tds_resident.cuh, in a translation unit of their own so that the families compile in parallel.
#include "tds_resident.cuh"

namespace tds {
TDS_FAMILY_DEFINE_NATIVE(f32, FamF32)
} // namespace tds
