// Closed-form integrals of G and F over one straight segment (App. D), as
// used by every near-field and dense kernel.
//
// For a target q and a segment p1 -> p2 of chord length c, let a = p1 - q,
// b = p2 - q.  The signed angle the segment subtends at q is
//     phi = atan2(a x b, a . b),
// and with n the right-hand unit normal of the segment direction,
//     int F dS = -phi / 2pi                       (Eq. 4 integrated)
//     int log|p - q| dS = ( s2 log|b|^2 - s1 log|a|^2 ) / 2 - c + (a x b / c) phi
// where s1 = a.d/c, s2 = b.d/c are the endpoints' coordinates along the
// chord (d = p2 - p1), and (a x b)/c is the signed offset of q from the
// chord's line.  int G dS = -(1/2pi) int log|p - q| dS.  Both are scaled
// by the segment's arc-length weight w (App. A).  When q lies on the
// segment (its own collocation segment), phi is replaced by 0: the
// principal value of Eq. 53, and the log form then equals Eq. 52.
#pragma once

#include <cuda_runtime.h>

namespace dc {

constexpr double kInv2Pi = 0.15915494309189533577;

__device__ __forceinline__ void seg_gf_f64(double qx, double qy, double x1, double y1,
                                           double x2, double y2, double w, bool own,
                                           double &G, double &F) {
    double ax = x1 - qx, ay = y1 - qy;
    double bx = x2 - qx, by = y2 - qy;
    double dx = x2 - x1, dy = y2 - y1;
    double ic = rsqrt(dx * dx + dy * dy);
    double c = (dx * dx + dy * dy) * ic;
    double cr = ax * by - ay * bx;
    double dt = ax * bx + ay * by;
    double phi = own ? 0.0 : atan2(cr, dt);
    double ra2 = ax * ax + ay * ay, rb2 = bx * bx + by * by;
    double s1 = (ax * dx + ay * dy) * ic, s2 = (bx * dx + by * dy) * ic;
    double la = (ra2 > 0.0) ? s1 * log(ra2) : 0.0;
    double lb = (rb2 > 0.0) ? s2 * log(rb2) : 0.0;
    double ilog = 0.5 * (lb - la) - c + cr * ic * phi;
    G = -w * kInv2Pi * ilog;
    F = -w * kInv2Pi * phi;
}

// int G dS / w of a segment far from q (at least a few chord lengths), in
// FP32 from a = p1 - q, b = p2 - q and d = p2 - p1 taken in FP64 and then
// rounded: the terms are smooth there.
__device__ __forceinline__ float seg_g_far_f32(double ax, double ay, double bx, double by, double dx, double dy) {
    const float fax = (float)ax, fay = (float)ay, fbx = (float)bx, fby = (float)by;
    const float fdx = (float)dx, fdy = (float)dy;
    const float c2 = fdx * fdx + fdy * fdy, ic = rsqrtf(c2), c = c2 * ic;
    const float cr = fax * fby - fay * fbx;
    const float phi = atan2f(cr, fax * fbx + fay * fby);
    const float la = (fax * fdx + fay * fdy) * ic * logf(fax * fax + fay * fay);
    const float lb = (fbx * fdx + fby * fdy) * ic * logf(fbx * fbx + fby * fby);
    return -(float)kInv2Pi * (0.5f * (lb - la) - c + cr * ic * phi);
}

// Whether segment (a, b, d as above) is within r chord lengths of q.
__device__ __forceinline__ bool seg_is_near(double ax, double ay, double bx, double by, double dx, double dy,
                                            double r) {
    const double h2 = r * r * (dx * dx + dy * dy);
    return ax * ax + ay * ay < h2 || bx * bx + by * by < h2;
}

// Unweighted parts of the same rule: ilog = int log|p - q| dS over the chord
// and phi = subtended angle (0 on the own segment).
__device__ __forceinline__ void seg_ilog_phi_f64(double qx, double qy, double x1, double y1,
                                                 double x2, double y2, bool own, double &ilog,
                                                 double &phi) {
    double ax = x1 - qx, ay = y1 - qy;
    double bx = x2 - qx, by = y2 - qy;
    double dx = x2 - x1, dy = y2 - y1;
    double ic = rsqrt(dx * dx + dy * dy);
    double c = (dx * dx + dy * dy) * ic;
    double cr = ax * by - ay * bx;
    double dt = ax * bx + ay * by;
    phi = own ? 0.0 : atan2(cr, dt);
    double ra2 = ax * ax + ay * ay, rb2 = bx * bx + by * by;
    double s1 = (ax * dx + ay * dy) * ic, s2 = (bx * dx + by * dy) * ic;
    double la = (ra2 > 0.0) ? s1 * log(ra2) : 0.0;
    double lb = (rb2 > 0.0) ? s2 * log(rb2) : 0.0;
    ilog = 0.5 * (lb - la) - c + cr * ic * phi;
}

}  // namespace dc
