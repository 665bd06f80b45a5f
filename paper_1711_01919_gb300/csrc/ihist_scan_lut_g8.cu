// ihist_scan_lut_g8.cu -- instantiations of the scan kernel for 8 bins per CTA
// that bin through a 256-entry value -> bin table (other bin structures).

#include "ihist_kernels.h"

namespace ihist {

namespace {
template <int MMAX>
ScanFn pick(bool tma, bool vec) {
  if (tma) return vec ? scan_kernel<8, MMAX, true, true, true> : scan_kernel<8, MMAX, true, false, true>;
  return vec ? scan_kernel<8, MMAX, false, true, true> : scan_kernel<8, MMAX, false, false, true>;
}
}  // namespace

ScanFn scan_fn_lut_g8(int mmax, bool tma, bool vec) {
  switch (mmax) {
    case 1: return pick<1>(tma, vec);
    case 2: return pick<2>(tma, vec);
    case 4: return pick<4>(tma, vec);
    case 8: return pick<8>(tma, vec);
    default: return nullptr;
  }
}

}  // namespace ihist
