// tds_fam_split.cu -- the split-precision FP64 (TrSplit<W>: float-pair recurrences) instantiations
// of the resident kernels of tds_resident.cuh, in a translation unit of their own so that the
// families compile in parallel.
#include "tds_resident.cuh"

namespace tds {
TDS_FAMILY_DEFINE(split, FamSplit)
} // namespace tds
