// Data shared between the kernel-build pipeline and its FFT passes.
#pragma once

#include "common.cuh"

namespace wproj {

// A batch of nb kernel boxes of side S being built.
struct BoxBatch {
  int S = 0;
  int nb = 0;
  const float2 *Au = nullptr;     // [nb][S] per-axis factor: KB tap polynomial x e^{2 pi i w l^2 / 2}
  const float2 *Av = nullptr;     // [nb][S]
  const int8_t *mode = nullptr;   // [nb] 0: separable phase only; 1: + FP32 remainder; 2: FP64 phase
  const float *wf = nullptr;      // [nb] w as float (remainder term)
  const double *wd = nullptr;     // [nb] w (FP64 phase path)
  const float *lsq = nullptr;     // [S] l_P^2 (float)
  const double *lcoord = nullptr; // [S] l_P (after clamping)
  float2 *K = nullptr;            // [nb][S][S] kernel values, natural order (offset s at s mod S)
  // direction-dependent screens (S = G): screens[bsid[b]] multiplies box b's samples;
  // screen index a holds offset a - S/2 (centred), the box sample P offset P or P - S
  const float2 *screens = nullptr;
  const int32_t *bsid = nullptr;
};

}  // namespace wproj
