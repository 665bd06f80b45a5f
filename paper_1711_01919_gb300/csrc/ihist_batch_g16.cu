// ihist_batch_g16.cu -- instantiations of the batched kernel for 16 bins per CTA.
// G = 16 keeps 64 accumulators per lane: built for up to 2 chunks per warp.
#include "ihist_kernels.h"

namespace ihist {

namespace {
template <int MMAX>
BatchFn pick(bool tma, bool vec) {
  if (tma) return vec ? batch_kernel<16, MMAX, true, true, false> : batch_kernel<16, MMAX, true, false, false>;
  return vec ? batch_kernel<16, MMAX, false, true, false> : batch_kernel<16, MMAX, false, false, false>;
}
}  // namespace

BatchFn batch_fn_g16(int mmax, bool tma, bool vec) {
  switch (mmax) {
    case 1: return pick<1>(tma, vec);
    case 2: return pick<2>(tma, vec);
    default: return nullptr;
  }
}

}  // namespace ihist
