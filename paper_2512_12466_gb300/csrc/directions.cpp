// Ray directions: HEALPix nested pixel centres (Gorski et al. 2005, the
// discretisation the adaptive ray tracer of Sec. 2.5 splits rays on), each
// component quantised to 2^-21 so the march can take every traversal
// decision with exact integer arithmetic. Built on the host once per level
// range and uploaded; the children of pixel p at level l are 4p..4p+3 at
// level l+1 (nested scheme).
//
// Compiled with -ffp-contract=off: the table must be the IEEE evaluation of
// the formulas below, so that it is the same on every host.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "rt_internal.h"

namespace nyx {

namespace {

// Base-face layout of the nested scheme: ring offset (in units of N_side)
// and phi offset (in units of pi/(4 nr)) of each of the 12 faces.
const int kFaceRing[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
const int kFacePhi[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

// Split a Z-order (Morton) index into its x (even bits) and y (odd bits).
void morton_split(int64_t m, int bits, int64_t* x, int64_t* y)
{
    int64_t a = 0, b = 0;
    for (int i = 0; i < bits; ++i) {
        a |= ((m >> (2 * i)) & 1) << i;
        b |= ((m >> (2 * i + 1)) & 1) << i;
    }
    *x = a;
    *y = b;
}

// Centre of nested pixel `pix` at resolution 2^level as (cos phi sin theta,
// sin phi sin theta, cos theta).
void pixel_centre(int level, int64_t pix, double v[3])
{
    const int64_t ns = int64_t(1) << level;
    const int face = int(pix / (ns * ns));
    int64_t fx, fy;
    morton_split(pix % (ns * ns), level, &fx, &fy);
    const int64_t ring = kFaceRing[face] * ns - fx - fy - 1;    // 1 .. 4 ns - 1 from the north pole

    int64_t nr;          // pixels per quarter ring
    int shifted;         // ring offset by half a pixel in phi
    double z, sin_t;
    if (ring < ns || ring > 3 * ns) {                           // polar caps
        nr = ring < ns ? ring : 4 * ns - ring;
        const double q = double(nr * nr) / double(3 * ns * ns);  // 1 - |z|
        z = ring < ns ? 1.0 - q : q - 1.0;
        sin_t = std::sqrt(q * (2.0 - q));
        shifted = 0;
    } else {                                                    // equatorial belt
        nr = ns;
        z = (double(2 * ns - ring) * 2.0) / double(3 * ns);
        sin_t = std::sqrt((1.0 - z) * (1.0 + z));
        shifted = int((ring - ns) & 1);
    }
    int64_t j = (kFacePhi[face] * nr + fx - fy + 1 + shifted) / 2;   // 1 .. 4 nr along the ring
    if (j > 4 * ns) j -= 4 * ns;
    if (j < 1) j += 4 * ns;
    const double phi = ((double(j) - 0.5 * double(shifted + 1)) * 1.5707963267948966) / double(nr);
    v[0] = sin_t * std::cos(phi);
    v[1] = sin_t * std::sin(phi);
    v[2] = z;
}

}  // namespace

int64_t healpix_level_offset(int level)
{
    // sum_{l < level} 12 * 4^l = 4 (4^level - 1)
    return 4 * ((int64_t(1) << (2 * level)) - 1);
}

void healpix_direction_table(int max_level, int4* out)
{
    const double scale = double(1 << kDirBits);
    for (int level = 0; level <= max_level; ++level) {
        const int64_t npix = 12 * (int64_t(1) << (2 * level));
        int4* row = out + healpix_level_offset(level);
        for (int64_t p = 0; p < npix; ++p) {
            double v[3];
            pixel_centre(level, p, v);
            int32_t c[3];
            int64_t norm2 = 0;
            for (int a = 0; a < 3; ++a) {
                const int32_t m = int32_t(std::floor(std::fabs(v[a]) * scale + 0.5));
                c[a] = v[a] < 0 ? -m : m;
                norm2 += int64_t(m) * m;
            }
            // |quantised direction| / 2^21, rounded to float for the FP32 march.
            const float nrm = float(std::sqrt(double(norm2)) / scale);
            int32_t nb;
            std::memcpy(&nb, &nrm, 4);
            row[p] = make_int4(c[0], c[1], c[2], nb);
        }
    }
}

}  // namespace nyx
