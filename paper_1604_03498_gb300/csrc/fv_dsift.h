// Dense SIFT plan shared by the dense-SIFT kernels and the PCA projection's
// gather path: per scale of the pyramid, the sizes, the descriptor grid, the
// x-pass / y-pass lattice and the offsets of each buffer within a frame.
#pragma once
#include <cstdint>

namespace fv {

constexpr int kMaxScales = 9;

struct DsScale {
    int Hs, Ws;
    float inv_s;      // 1 / s
    int ny, nx;       // descriptor grid
    int Tx;           // lattice columns b/2 + S t, t < Tx
    int Ty;           // lattice rows b/2 + S m, m < Ty
    int64_t img_off;  // floats into a frame's pyramid
    int64_t tmp_off;  // floats into a frame's x-pass buffer [8][Hs][Tx]
    int64_t yp_off;   // floats into a frame's y-pass buffer [Ty][Tx][8]
    int64_t lat_off;  // first y-pass thread (lattice point) of the scale within a frame
    int64_t desc_off; // first descriptor of the scale within a frame
    int64_t pix_off;  // first x-pass thread of the scale within a frame
};

struct DsPlan {
    int n, b, S;
    DsScale s[kMaxScales];
    int64_t pyr, tmp, ndesc, npix;   // per-frame totals (pyramid floats, x-pass floats, descriptors, x-pass points)
    int64_t yp, nlat;                // per-frame totals (y-pass floats, lattice points)
};

}  // namespace fv
