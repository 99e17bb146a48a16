// hot_box.cuh -- the field of a uniform box, for background subtraction (Sec. "Background
// Subtraction": the background of the near field is removed by the analytic force inside
// and around a uniform cube).
//
// Closed form (Waldvogel): with (u, v, w) a corner of the box relative to the field point,
// r = |(u, v, w)|, and s = +1 / -1 for an even / odd number of lower limits,
//   int dV / r            = sum_corners s F,
//   F = u v ln(w + r) + v w ln(u + r) + w u ln(v + r)
//       - (u^2 atan(v w / (u r)) + v^2 atan(w u / (v r)) + w^2 atan(u v / (w r))) / 2,
//   int (x' - x)_x / r^3 dV = -sum_corners s (v ln(w + r) + w ln(v + r) - u atan(v w / (u r))),
// and cyclically for y, z.  ln(a + r) is taken as ln((b^2 + c^2) / (r - a)) for a < 0 (no
// cancellation), and a term whose factor vanishes (a corner on an edge or face through the
// point) as 0.  The eight corner terms cancel to the field, so the form is for points
// within a few box sizes (farther boxes are expanded); the including file evaluates it in
// float64.
//
// The including file supplies hb_log, hb_atan, hb_sqrt and hb_div for T (the device's log,
// atan and sqrt in CUDA code, a division of at most a few units in the last place for
// float32, whose terms then move by about 1e-7 of their size; std:: versions and exact
// division where the header is compiled for the host).
#pragma once

// ln(a + r), r = |(a, b, c)|, bc2 = b^2 + c^2; 0 where a + r vanishes
template <class T>
__device__ __forceinline__ T hb_log_plus_r(T a, T r, T bc2)
{
    if (a >= T(0)) return a + r > T(0) ? hb_log(a + r) : T(0);
    return bc2 > T(0) ? hb_log(hb_div(bc2, r - a)) : T(0);
}

// atan(v w / (u r)); 0 where u = 0 (its factor u or u^2 then vanishes)
template <class T>
__device__ __forceinline__ T hb_atan_term(T u, T v, T w, T r)
{
    return u != T(0) ? hb_atan(hb_div(v * w, u * r)) : T(0);
}

// Adds to (ax, ay, az) the acceleration G rho int (x' - p) / |x' - p|^3 dV and to phi the
// potential -G rho int dV / |x' - p| of the box [lo, hi] of density rho (Grho = G rho) at
// the point p.
template <class T>
__device__ __forceinline__ void box_field(T px, T py, T pz, const T (&lo)[3], const T (&hi)[3], T Grho, T &ax, T &ay,
                                          T &az, T &phi)
{
    T sx = T(0), sy = T(0), sz = T(0), sp = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int cx = (k >> 2) & 1, cy = (k >> 1) & 1, cz = k & 1;
        const T sgn = ((3 - cx - cy - cz) & 1) ? T(-1) : T(1);  // (-1)^(number of lower limits)
        const T u = (cx ? hi[0] : lo[0]) - px;
        const T v = (cy ? hi[1] : lo[1]) - py;
        const T w = (cz ? hi[2] : lo[2]) - pz;
        const T u2 = u * u, v2 = v * v, w2 = w * w;
        const T r = hb_sqrt(u2 + v2 + w2);
        const T lu = hb_log_plus_r(u, r, v2 + w2);
        const T lv = hb_log_plus_r(v, r, w2 + u2);
        const T lw = hb_log_plus_r(w, r, u2 + v2);
        const T tu = hb_atan_term(u, v, w, r);
        const T tv = hb_atan_term(v, w, u, r);
        const T tw = hb_atan_term(w, u, v, r);
        const T F = u * v * lw + v * w * lu + w * u * lv - T(0.5) * (u2 * tu + v2 * tv + w2 * tw);
        sp += sgn * F;
        sx -= sgn * (v * lw + w * lv - u * tu);
        sy -= sgn * (w * lu + u * lw - v * tv);
        sz -= sgn * (u * lv + v * lu - w * tw);
    }
    ax += Grho * sx;
    ay += Grho * sy;
    az += Grho * sz;
    phi -= Grho * sp;
}
