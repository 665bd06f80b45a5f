// ihist_kernels.h -- host-visible handles of the scan-kernel instantiations.
// Each bins-per-CTA value G is compiled in its own translation unit
// (ihist_scan_g<G>.cu) so the instantiations build in parallel.
#pragma once

#include <cuda.h>

#include "ihist_scan.cuh"

namespace ihist {

using ScanFn = void (*)(FrameDesc, const CUtensorMap, Ctrl *, unsigned long long);
using BatchFn = void (*)(const FrameDesc *, const CUtensorMap *, const unsigned int *, int, int, int, int,
                         Ctrl *, unsigned long long);

// Kernel for (G, MMAX = chunks-per-warp bound, TMA input staging, 16-byte
// output stores); nullptr if that combination is not built.
ScanFn scan_fn_g4(int mmax, bool tma, bool vec);
ScanFn scan_fn_g8(int mmax, bool tma, bool vec);
ScanFn scan_fn_g16(int mmax, bool tma, bool vec);
ScanFn scan_fn_lut_g4(int mmax, bool tma, bool vec);  // binning through a value -> bin table
ScanFn scan_fn_lut_g8(int mmax, bool tma, bool vec);
BatchFn batch_fn_g4(int mmax, bool tma, bool vec);
BatchFn batch_fn_g8(int mmax, bool tma, bool vec);
BatchFn batch_fn_g16(int mmax, bool tma, bool vec);  // mmax <= 2
BatchFn batch_fn_lut_g4(int mmax, bool tma, bool vec);  // per-frame value -> bin tables
BatchFn batch_fn_lut_g8(int mmax, bool tma, bool vec);

inline ScanFn scan_fn(int G, int mmax, bool tma, bool vec, bool lut = false) {
  if (lut) return G == 4 ? scan_fn_lut_g4(mmax, tma, vec) : G == 8 ? scan_fn_lut_g8(mmax, tma, vec) : nullptr;
  switch (G) {
    case 4: return scan_fn_g4(mmax, tma, vec);
    case 8: return scan_fn_g8(mmax, tma, vec);
    case 16: return scan_fn_g16(mmax, tma, vec);
    default: return nullptr;
  }
}

inline BatchFn batch_fn(int G, int mmax, bool tma, bool vec, bool lut = false) {
  if (lut) return G == 4 ? batch_fn_lut_g4(mmax, tma, vec) : G == 8 ? batch_fn_lut_g8(mmax, tma, vec) : nullptr;
  switch (G) {
    case 4: return batch_fn_g4(mmax, tma, vec);
    case 8: return batch_fn_g8(mmax, tma, vec);
    case 16: return batch_fn_g16(mmax, tma, vec);
    default: return nullptr;
  }
}

}  // namespace ihist
