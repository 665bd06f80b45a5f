// ihist_scan_g8.cu -- instantiations of the scan kernel for 8 bins per CTA.

#include "ihist_kernels.h"

namespace ihist {

namespace {
template <int MMAX>
ScanFn pick(bool tma, bool vec) {
  if (tma) return vec ? scan_kernel<8, MMAX, true, true, false> : scan_kernel<8, MMAX, true, false, false>;
  return vec ? scan_kernel<8, MMAX, false, true, false> : scan_kernel<8, MMAX, false, false, false>;
}
}  // namespace

ScanFn scan_fn_g8(int mmax, bool tma, bool vec) {
  switch (mmax) {
    case 1: return pick<1>(tma, vec);
    case 2: return pick<2>(tma, vec);
    case 4: return pick<4>(tma, vec);
    case 8: return pick<8>(tma, vec);
    default: return nullptr;
  }
}

}  // namespace ihist
