// ihist_scan_g16.cu -- instantiations of the scan kernel for 16 bins per CTA.
// G = 16 keeps 64 accumulators per lane: built for up to 2 chunks per warp.
#include "ihist_kernels.h"

namespace ihist {

namespace {
template <int MMAX>
ScanFn pick(bool tma, bool vec) {
  if (tma) return vec ? scan_kernel<16, MMAX, true, true, false> : scan_kernel<16, MMAX, true, false, false>;
  return vec ? scan_kernel<16, MMAX, false, true, false> : scan_kernel<16, MMAX, false, false, false>;
}
}  // namespace

ScanFn scan_fn_g16(int mmax, bool tma, bool vec) {
  switch (mmax) {
    case 1: return pick<1>(tma, vec);
    case 2: return pick<2>(tma, vec);
    default: return nullptr;
  }
}

}  // namespace ihist
