// tds_fam_f64.cu -- the native FP64 (TrNative<double, W>) instantiations of the resident kernels of
// tds_resident.cuh, in a translation unit of their own so that the families compile in parallel.
#include "tds_resident.cuh"

namespace tds {
TDS_FAMILY_DEFINE_NATIVE(f64, FamF64)
} // namespace tds
