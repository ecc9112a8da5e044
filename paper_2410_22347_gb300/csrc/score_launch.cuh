// score_launch.cuh -- maps a runtime scoring configuration (lanes per candidate G, row
// pipelining) and a row width onto the compile-time kernel instantiation.
//
// For a row of nch 16-byte chunks and G lanes per candidate, every lane loads
// NCH = ceil(nch / G) chunks.  Gather modes: 0 = row loads into registers, 1 = the same with
// the next candidate's loads issued before the current dot (pipelined), 2 = bulk copies of
// whole rows into shared memory (score_bulk.cuh; stand-alone kernel only).  Instantiated:
// NCH in {1..6, 8, 10} for modes 0 and 2, NCH <= 5 for mode 1; G in the store type's three
// group sizes plus 32.  Each (store type, kernel, mode) is compiled in its own translation
// unit (score_<type>_<plain|fused>_m<mode>.cu).
#pragma once

#include "kernels.cuh"
#include "score_dev.cuh"

namespace glv {

// Group sizes offered per store type: the default G0 and its half and double.
template <int DT>
struct Groups {
  static constexpr int G0 = default_group<DT>();
  static constexpr int kLo = G0 > 1 ? G0 / 2 : 1;
  static constexpr int kHi = G0 * 2;
};

inline bool nch_supported(int n, int mode) {
  if (mode == 1) return n >= 1 && n <= 5;
  return (n >= 1 && n <= 6) || n == 8 || n == 10;
}

// Whether a configuration (G, mode) is instantiated for store type DT.
template <int DT>
inline bool group_supported(int G, int mode) {
  (void)mode;
  return G == Groups<DT>::kLo || G == Groups<DT>::G0 || G == Groups<DT>::kHi || G == 32;
}

// Smallest instantiated NCH >= n (extra slots are predicated off).
inline int round_nch(int n, int mode) {
  while (n <= 10 && !nch_supported(n, mode)) ++n;
  return n;
}

template <int DT, int G, int MODE, class F>
cudaError_t dispatch_nch_mode(int n, F& f) {
  switch (n) {
    case 1: return f.template go<DT, G, 1, MODE>();
    case 2: return f.template go<DT, G, 2, MODE>();
    case 3: return f.template go<DT, G, 3, MODE>();
    case 4: return f.template go<DT, G, 4, MODE>();
    case 5: return f.template go<DT, G, 5, MODE>();
    default: break;
  }
  if constexpr (MODE != 1) {
    switch (n) {
      case 6: return f.template go<DT, G, 6, MODE>();
      case 8: return f.template go<DT, G, 8, MODE>();
      case 10: return f.template go<DT, G, 10, MODE>();
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

// Call f.template go<DT, G, NCH, MODE>() for the lane count G of one gather mode.
template <int DT, int MODE, class F>
cudaError_t dispatch_score_mode(int G, int nch, F& f) {
  using Gs = Groups<DT>;
  const int n = round_nch((nch + G - 1) / G, MODE);
  if (G == Gs::kLo) return dispatch_nch_mode<DT, Gs::kLo, MODE>(n, f);
  if (G == Gs::G0) return dispatch_nch_mode<DT, Gs::G0, MODE>(n, f);
  if (G == Gs::kHi) return dispatch_nch_mode<DT, Gs::kHi, MODE>(n, f);
  if (G == 32) return dispatch_nch_mode<DT, 32, MODE>(n, f);
  return cudaErrorInvalidValue;
}

// The wide fused kernel (512 threads) is instantiated for the two smaller group sizes of a
// store type, register loads only.
template <int DT>
inline bool wide_group_supported(int G) {
  return G == Groups<DT>::kLo || G == Groups<DT>::G0;
}

template <int DT, class F>
cudaError_t dispatch_score_wide(int G, int nch, F& f) {
  using Gs = Groups<DT>;
  const int n = round_nch((nch + G - 1) / G, 0);
  if (G == Gs::kLo) return dispatch_nch_mode<DT, Gs::kLo, 0>(n, f);
  if (G == Gs::G0) return dispatch_nch_mode<DT, Gs::G0, 0>(n, f);
  return cudaErrorInvalidValue;
}

// Effective configuration for a row of nch chunks: the tuned choice if it can serve the
// row, else the default group (or 32 lanes for wide rows) with register loads.
// Lanes per candidate, gather mode, the shared-memory carveout cap in KB (0 = the driver's
// choice) and the fused call's schedule.  The driver sizes the shared-memory / L1 split for the kernel's full
// occupancy, and the L1 that is left stages the rows in flight, so a smaller carveout (fewer
// CTAs, more L1) can gather faster; which one wins depends on the store, d and C.
struct ScoreConfig {
  int G;
  int mode;
  int carve_kb = 0;
  int sched = 1;  // fused call, bit 0: planned work items (chunked long lists), else one CTA per
                  // query; bit 1: wide CTAs (512 threads, register loads)
};

template <int DT>
ScoreConfig effective_config(int nch, int tuned_G, int tuned_mode) {
  auto fits = [&](int G, int mode) { return G > 0 && round_nch((nch + G - 1) / G, mode) <= 10; };
  if (tuned_G > 0 && group_supported<DT>(tuned_G, tuned_mode) && fits(tuned_G, tuned_mode))
    return {tuned_G, tuned_mode};
  if (fits(Groups<DT>::G0, 0)) return {Groups<DT>::G0, 0};
  if (fits(Groups<DT>::kHi, 0)) return {Groups<DT>::kHi, 0};
  return {32, 0};
}

// The library-default configuration only (register gather), for kernels that are not tuned.
template <int DT, class F>
cudaError_t dispatch_score_default(int nch, F& f) {
  const ScoreConfig c = effective_config<DT>(nch, 0, 0);
  const int n = round_nch((nch + c.G - 1) / c.G, 0);
  if (c.G == Groups<DT>::G0) return dispatch_nch_mode<DT, Groups<DT>::G0, 0>(n, f);
  if (c.G == Groups<DT>::kHi) return dispatch_nch_mode<DT, Groups<DT>::kHi, 0>(n, f);
  return dispatch_nch_mode<DT, 32, 0>(n, f);
}

}  // namespace glv
