// Host construction of the normal-bin candidate table used by the query kernel.
//
// The query bins the contact-surface normal m by argmax_b d_b . m (first
// maximum).  The kernel looks m up in a cube map (major axis -> face, the other
// two components over the major one -> (u, v) cell) and evaluates only the bins
// listed for that cell.  A bin is listed if it can be the argmax for SOME unit
// direction of the (slightly enlarged) cell: with c the cell's centre
// direction and delta the largest chord from c to the cell's corners, every
// direction x of the cell has |d_b . x - d_b . c| <= delta, so the true argmax
// b* satisfies d_b* . c >= max_b d_b . c - 2 delta.  Listing every b above that
// bound (minus a float margin) keeps b* and every bin tied with it; evaluated in
// ascending order with a strict comparison they give the full-scan answer.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "cf_internal.cuh"

namespace cf {

namespace {
void face_dir(int face, double u, double v, double out[3]) {
    const int ax = face / 2;
    const double sgn = (face % 2 == 0) ? 1.0 : -1.0;
    const int a = ax == 0 ? 1 : 0, b = ax == 2 ? 1 : 2;
    double x[3];
    x[ax] = sgn;
    x[a] = u;
    x[b] = v;
    const double n = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    for (int i = 0; i < 3; ++i) out[i] = x[i] / n;
}
}  // namespace

int build_bin_candidates(const float *dirs, int B, uint32_t *table) {
    const double margin_uv = 1e-4;   // cell enlargement (covers the kernel's float cell choice)
    const double margin_dot = 1e-5;  // covers float dot-product rounding on both sides
    int worst = 0;
    for (int face = 0; face < 6; ++face) {
        for (int iu = 0; iu < kCandG; ++iu) {
            for (int iv = 0; iv < kCandG; ++iv) {
                const double u0 = -1.0 + 2.0 * iu / kCandG - margin_uv, u1 = -1.0 + 2.0 * (iu + 1) / kCandG + margin_uv;
                const double v0 = -1.0 + 2.0 * iv / kCandG - margin_uv, v1 = -1.0 + 2.0 * (iv + 1) / kCandG + margin_uv;
                double c[3];
                face_dir(face, 0.5 * (u0 + u1), 0.5 * (v0 + v1), c);
                double delta = 0.0;
                const double us[2] = {u0, u1}, vs[2] = {v0, v1};
                for (double uu : us)
                    for (double vv : vs) {
                        double x[3];
                        face_dir(face, uu, vv, x);
                        const double dx = x[0] - c[0], dy = x[1] - c[1], dz = x[2] - c[2];
                        delta = std::max(delta, sqrt(dx * dx + dy * dy + dz * dz));
                    }
                std::vector<double> s(B);
                double best = -INFINITY;
                for (int b = 0; b < B; ++b) {
                    s[b] = (double)dirs[3 * b] * c[0] + (double)dirs[3 * b + 1] * c[1] + (double)dirs[3 * b + 2] * c[2];
                    best = std::max(best, s[b]);
                }
                std::vector<int> cand;
                for (int b = 0; b < B; ++b)
                    if (s[b] >= best - 2.0 * delta - margin_dot) cand.push_back(b);
                worst = std::max(worst, (int)cand.size());
                uint32_t word = 0;
                const int n = std::min((int)cand.size(), 4);
                for (int i = 0; i < n; ++i) word |= (uint32_t)(cand[i] & 63) << (6 * i);
                word |= (uint32_t)n << 24;
                table[(face * kCandG + iu) * kCandG + iv] = word;
            }
        }
    }
    return worst;
}

}  // namespace cf
