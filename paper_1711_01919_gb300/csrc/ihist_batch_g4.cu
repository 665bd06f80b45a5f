// ihist_batch_g4.cu -- instantiations of the batched kernel for 4 bins per CTA.
#include "ihist_kernels.h"

namespace ihist {

namespace {
template <int MMAX>
BatchFn pick(bool tma, bool vec) {
  if (tma) return vec ? batch_kernel<4, MMAX, true, true, false> : batch_kernel<4, MMAX, true, false, false>;
  return vec ? batch_kernel<4, MMAX, false, true, false> : batch_kernel<4, MMAX, false, false, false>;
}
}  // namespace

BatchFn batch_fn_g4(int mmax, bool tma, bool vec) {
  switch (mmax) {
    case 1: return pick<1>(tma, vec);
    case 2: return pick<2>(tma, vec);
    case 4: return pick<4>(tma, vec);
    default: return nullptr;
  }
}

}  // namespace ihist
