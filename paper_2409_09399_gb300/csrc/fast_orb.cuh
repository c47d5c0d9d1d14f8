// fast_orb.cuh -- FP32 orbital values (and gradients) for the tensor-core
// producers: no per-orbital local arrays, species data in shared memory, the
// radial data of two adjacent knots per radial function from a compact FP32
// knot table, each orbital handed to a callback as soon as it is formed.
//
// phi_{l m}(d) = u(r) S_lm(d), u = R(r) / r^l, with R the cubic Hermite
// interpolant on the knot interval [k, k+1] (t = r/dr - k):
//   R = y_k h00(t) + y_k+1 h01(t) + m_k h10(t) + m_k+1 h11(t),  m = dr R'(knot),
// the same cubic as the oracle's, and S_lm the real solid harmonics
// (normalised Y_lm, no Condon-Shortley phase).  The knot table holds
// (y_k, m_k) as two FP32 words per knot and radial function: half the bytes of
// a per-interval power-basis table, so that more of it stays in L1.
// grad phi = u'(r) (d / r) S_lm + u grad S_lm, u' = (R' - l R / r) / r^l.
#pragma once

#include <type_traits>

#include "gint_impl.cuh"

namespace gint {

// Knot-table loads with L1 eviction priority "last": the table is the one
// global data set that every producer reads again and again (streaming data
// such as V and the pair tables is loaded with ld_stream_* and not kept in L1).
__device__ __forceinline__ float2 ld_knot(const float2* p) {
    float2 v;
    asm("ld.global.nc.L1::evict_last.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_stream_f64(const double* p) {
    double v;
    asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_stream_s32(const int* p) {
    int v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

struct SpeciesFast {
    int n_radial;
    int n_int;
    int lmax;
    int nw;
    float rc2;
    float inv_dr;
    int knot2;            // offset of the species' knot table in float2 units
    int rad_l[kMaxRadial];
    int orb_base[kMaxRadial];  // first orbital of each radial function
    signed char qe[kMaxNw];    // fixed-point quantum exponent of each orbital (|phi| <= 127 * 2^qe)
    signed char qeu[kMaxNw];   // the same for the unnormalised orbital phi / ylm_norm
    int dzp;                   // 1: five radial functions with l = 0, 0, 1, 1, 2 (s, s', p, p', d)
};

__device__ __forceinline__ void species_fast_from(const SpeciesDev& s, SpeciesFast& f) {
    f.n_radial = s.n_radial;
    f.n_int = s.n_int;
    f.lmax = s.lmax;
    f.nw = s.n_orb;
    f.rc2 = s.rc_f * s.rc_f;
    f.inv_dr = s.inv_dr_f;
    f.knot2 = (int)s.knot_off;
    for (int j = 0; j < kMaxRadial; ++j) { f.rad_l[j] = j < s.n_radial ? s.rad_l[j] : 0; f.orb_base[j] = 0; }
    for (int o = 0; o < kMaxNw; ++o) {
        f.qe[o] = o < s.n_orb ? s.orb_qe[o] : 0;
        f.qeu[o] = o < s.n_orb ? s.orb_qeu[o] : 0;
    }
    // orbital order: l ascending, radial functions in input order, m = -l..l
    int o = 0;
    for (int l = 0; l <= kMaxL; ++l)
        for (int j = 0; j < s.n_radial; ++j)
            if (s.rad_l[j] == l) { f.orb_base[j] = o; o += 2 * l + 1; }
    f.dzp = s.n_radial == 5 && f.rad_l[0] == 0 && f.rad_l[1] == 0 && f.rad_l[2] == 1 && f.rad_l[3] == 1 &&
            f.rad_l[4] == 2;
}

// The orbitals of one radial function of angular momentum L at displacement d:
// put(o + m, phi, grad phi) for m = 0 .. 2L, from u = R / r^L and a = u' / r (the
// gradient arguments are meaningful only with kGrad).
template <int L, bool kGrad, typename Put>
__device__ __forceinline__ void put_l(int o, float u, float a, float dx, float dy, float dz, Put&& put) {
    const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
    if (L == 0) {
        const float k00 = 0.28209479177387814f;
        put(o, u * k00, a * k00 * dx, a * k00 * dy, a * k00 * dz);
    } else if (L == 1) {
        const float k1 = 0.48860251190291992f;
        const float sy = k1 * dy, sz = k1 * dz, sx = k1 * dx;
        put(o + 0, u * sy, a * sy * dx, a * sy * dy + u * k1, a * sy * dz);
        put(o + 1, u * sz, a * sz * dx, a * sz * dy, a * sz * dz + u * k1);
        put(o + 2, u * sx, a * sx * dx + u * k1, a * sx * dy, a * sx * dz);
    } else if (L == 2) {
        const float k2a = 1.0925484305920792f, k2b = 0.31539156525252005f, k2c = 0.54627421529603959f;
        const float s4 = k2a * dx * dy, s5 = k2a * dy * dz, s6 = k2b * (2.f * zz - xx - yy);
        const float s7 = k2a * dx * dz, s8 = k2c * (xx - yy);
        put(o + 0, u * s4, a * s4 * dx + u * k2a * dy, a * s4 * dy + u * k2a * dx, a * s4 * dz);
        put(o + 1, u * s5, a * s5 * dx, a * s5 * dy + u * k2a * dz, a * s5 * dz + u * k2a * dy);
        put(o + 2, u * s6, a * s6 * dx - u * 2.f * k2b * dx, a * s6 * dy - u * 2.f * k2b * dy,
            a * s6 * dz + u * 4.f * k2b * dz);
        put(o + 3, u * s7, a * s7 * dx + u * k2a * dz, a * s7 * dy, a * s7 * dz + u * k2a * dx);
        put(o + 4, u * s8, a * s8 * dx + u * 2.f * k2c * dx, a * s8 * dy - u * 2.f * k2c * dy, a * s8 * dz);
    } else {
        const float k3a = 0.59004358992664352f, k3b = 2.8906114426405538f, k3c = 0.45704579946446572f;
        const float k3d = 0.37317633259011540f, k3e = 1.4453057213202769f;
        const float q5 = 4.f * zz - xx - yy;
        const float s9 = k3a * dy * (3.f * xx - yy), s10 = k3b * dx * dy * dz, s11 = k3c * dy * q5;
        const float s12 = k3d * dz * (2.f * zz - 3.f * xx - 3.f * yy), s13 = k3c * dx * q5;
        const float s14 = k3e * dz * (xx - yy), s15 = k3a * dx * (xx - 3.f * yy);
        put(o + 0, u * s9, a * s9 * dx + u * k3a * 6.f * dx * dy, a * s9 * dy + u * k3a * 3.f * (xx - yy), a * s9 * dz);
        put(o + 1, u * s10, a * s10 * dx + u * k3b * dy * dz, a * s10 * dy + u * k3b * dx * dz,
            a * s10 * dz + u * k3b * dx * dy);
        put(o + 2, u * s11, a * s11 * dx - u * k3c * 2.f * dx * dy, a * s11 * dy + u * k3c * (q5 - 2.f * yy),
            a * s11 * dz + u * k3c * 8.f * dy * dz);
        put(o + 3, u * s12, a * s12 * dx - u * k3d * 6.f * dx * dz, a * s12 * dy - u * k3d * 6.f * dy * dz,
            a * s12 * dz + u * k3d * (6.f * zz - 3.f * xx - 3.f * yy));
        put(o + 4, u * s13, a * s13 * dx + u * k3c * (q5 - 2.f * xx), a * s13 * dy - u * k3c * 2.f * dx * dy,
            a * s13 * dz + u * k3c * 8.f * dx * dz);
        put(o + 5, u * s14, a * s14 * dx + u * k3e * 2.f * dx * dz, a * s14 * dy - u * k3e * 2.f * dy * dz,
            a * s14 * dz + u * k3e * (xx - yy));
        put(o + 6, u * s15, a * s15 * dx + u * k3a * 3.f * (xx - yy), a * s15 * dy - u * k3a * 6.f * dx * dy,
            a * s15 * dz);
    }
}

// Calls put(o, phi, gx, gy, gz) for every orbital o of the species at
// displacement d (the gradient arguments are meaningful only with kGrad);
// returns false (no calls) when |d| >= rc.  Species of the s, s', p, p', d
// shape take an unrolled path that loads the knots of all five radial
// functions at once.  pre() runs once the first knot loads are issued and
// before the first put.
template <bool kGrad, typename Put, typename Pre>
__device__ __forceinline__ bool orbitals_fast(const SpeciesFast& s, const float2* __restrict__ knot, float dx,
                                              float dy, float dz, Put&& put, Pre&& pre) {
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= s.rc2) return false;
    const bool tiny = r2 < 1e-20f;
    const float r = sqrtf(r2);
    const float rinv = tiny ? 0.f : 1.f / r;
    float x = r * s.inv_dr;
    int k = (int)x;
    k = min(k, s.n_int - 1);
    const float t = x - (float)k;
    // cubic Hermite basis at t and (for the gradient) its t-derivative
    const float t1 = 1.f - t, tt = t * t;
    const float h00 = (1.f + 2.f * t) * t1 * t1, h10 = t * t1 * t1, h01 = tt * (3.f - 2.f * t), h11 = tt * (t - 1.f);
    const float g00 = 6.f * t * (t - 1.f), g10 = t1 * (1.f - 3.f * t), g11 = t * (3.f * t - 2.f);
    const int nr = s.n_radial;
    const float2* kn = knot + s.knot2 + k * nr;
    // the orbitals of radial function j (angular momentum l, first orbital o) from the
    // (R, dr R') pairs y0, y1 at knots k, k + 1
    auto radial = [&](auto lc, int o, float2 y0, float2 y1) {
        constexpr int l = decltype(lc)::value;
        const float R = y0.x * h00 + y1.x * h01 + y0.y * h10 + y1.y * h11;
        float dR = 0.f;
        if (kGrad) dR = ((y0.x - y1.x) * g00 + y0.y * g10 + y1.y * g11) * s.inv_dr;
        if (tiny) {
            // limits at the atom centre: phi = R(0) Y00 for l = 0, zero for l >= 1;
            // grad phi = R'(0) grad S_1m for l = 1, zero otherwise (y0.y / dr = R'(0))
            const float k00 = 0.28209479177387814f, k1 = 0.48860251190291992f;
            if (l == 0) {
                put(o, R * k00, 0.f, 0.f, 0.f);
            } else if (l == 1) {
                const float gl = y0.y * s.inv_dr * k1;
                put(o + 0, 0.f, 0.f, gl, 0.f);
                put(o + 1, 0.f, 0.f, 0.f, gl);
                put(o + 2, 0.f, gl, 0.f, 0.f);
            } else {
                for (int m = 0; m < 2 * l + 1; ++m) put(o + m, 0.f, 0.f, 0.f, 0.f);
            }
            return;
        }
        float rl = 1.f;
        for (int q = 0; q < l; ++q) rl *= rinv;
        const float u = R * rl;
        const float a = kGrad ? (dR - (float)l * R * rinv) * rl * rinv : 0.f;  // u'/r
        put_l<l, kGrad>(o, u, a, dx, dy, dz, put);
    };
    using L0 = std::integral_constant<int, 0>;
    using L1 = std::integral_constant<int, 1>;
    using L2 = std::integral_constant<int, 2>;
    using L3 = std::integral_constant<int, 3>;
    if (s.dzp) {
        float2 y0[5], y1[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) { y0[j] = ld_knot(kn + j); y1[j] = ld_knot(kn + 5 + j); }
        pre();  // the knot loads are in flight
        radial(L0{}, 0, y0[0], y1[0]);
        radial(L0{}, 1, y0[1], y1[1]);
        radial(L1{}, 2, y0[2], y1[2]);
        radial(L1{}, 5, y0[3], y1[3]);
        radial(L2{}, 8, y0[4], y1[4]);
        return true;
    }
    // (R, dr R') at knots k, k + 1; those of radial function j + 1 are loaded before the
    // values of j are formed, so their latency overlaps that work
    float2 y0n = make_float2(0.f, 0.f), y1n = y0n;
    if (nr > 0) { y0n = ld_knot(kn); y1n = ld_knot(kn + nr); }
    pre();
    for (int j = 0; j < nr; ++j) {
        const float2 y0 = y0n, y1 = y1n;
        if (j + 1 < nr) { y0n = ld_knot(kn + j + 1); y1n = ld_knot(kn + nr + j + 1); }
        const int l = s.rad_l[j];
        const int o = s.orb_base[j];
        if (l == 0) radial(L0{}, o, y0, y1);
        else if (l == 1) radial(L1{}, o, y0, y1);
        else if (l == 2) radial(L2{}, o, y0, y1);
        else radial(L3{}, o, y0, y1);
    }
    return true;
}

template <bool kGrad, typename Put>
__device__ __forceinline__ bool orbitals_fast(const SpeciesFast& s, const float2* __restrict__ knot, float dx,
                                              float dy, float dz, Put&& put) {
    return orbitals_fast<kGrad>(s, knot, dx, dy, dz, put, [] {});
}

}  // namespace gint

namespace gint {

// The orbitals of one radial function of angular momentum L at two points a, b:
// put2(o + m, value at a, value at b) for m = 0 .. 2L, from the radial parts ua, ub
// (already divided by r^L).  kNorm = false leaves out the harmonic normalisation.
template <int L, bool kNorm, typename Put2>
__device__ __forceinline__ void put_l2(int o, float ua, float ub, float ax, float ay, float az, float bx, float by,
                                       float bz, Put2&& put2) {
    if (L == 0) {
        const float k00 = kNorm ? 0.28209479177387814f : 1.f;
        put2(o, ua * k00, ub * k00);
    } else if (L == 1) {
        const float k1 = kNorm ? 0.48860251190291992f : 1.f;
        put2(o + 0, ua * k1 * ay, ub * k1 * by);
        put2(o + 1, ua * k1 * az, ub * k1 * bz);
        put2(o + 2, ua * k1 * ax, ub * k1 * bx);
    } else if (L == 2) {
        const float k2a = kNorm ? 1.0925484305920792f : 1.f, k2b = kNorm ? 0.31539156525252005f : 1.f;
        const float k2c = kNorm ? 0.54627421529603959f : 1.f;
        put2(o + 0, ua * k2a * ax * ay, ub * k2a * bx * by);
        put2(o + 1, ua * k2a * ay * az, ub * k2a * by * bz);
        put2(o + 2, ua * k2b * (2.f * az * az - ax * ax - ay * ay), ub * k2b * (2.f * bz * bz - bx * bx - by * by));
        put2(o + 3, ua * k2a * ax * az, ub * k2a * bx * bz);
        put2(o + 4, ua * k2c * (ax * ax - ay * ay), ub * k2c * (bx * bx - by * by));
    } else {
        const float k3a = kNorm ? 0.59004358992664352f : 1.f, k3b = kNorm ? 2.8906114426405538f : 1.f;
        const float k3c = kNorm ? 0.45704579946446572f : 1.f;
        const float k3d = kNorm ? 0.37317633259011540f : 1.f, k3e = kNorm ? 1.4453057213202769f : 1.f;
        const float xxa = ax * ax, yya = ay * ay, zza = az * az, xxb = bx * bx, yyb = by * by, zzb = bz * bz;
        const float wa = 4.f * zza - xxa - yya, wb = 4.f * zzb - xxb - yyb;
        put2(o + 0, ua * k3a * ay * (3.f * xxa - yya), ub * k3a * by * (3.f * xxb - yyb));
        put2(o + 1, ua * k3b * ax * ay * az, ub * k3b * bx * by * bz);
        put2(o + 2, ua * k3c * ay * wa, ub * k3c * by * wb);
        put2(o + 3, ua * k3d * az * (2.f * zza - 3.f * xxa - 3.f * yya), ub * k3d * bz * (2.f * zzb - 3.f * xxb - 3.f * yyb));
        put2(o + 4, ua * k3c * ax * wa, ub * k3c * bx * wb);
        put2(o + 5, ua * k3e * az * (xxa - yya), ub * k3e * bz * (xxb - yyb));
        put2(o + 6, ua * k3a * ax * (xxa - 3.f * yya), ub * k3a * bx * (xxb - 3.f * yyb));
    }
}

// Orbital values of one atom image at two points: put2(o, v0, v1) for every
// orbital o; a point outside the cutoff contributes 0.  Returns false (no
// calls) when both points are outside.  Same functions as orbitals_fast; with
// kNorm = false the harmonic normalisation ylm_norm(l, m) is left out (the
// caller applies it in FP64).  Species of the s, s', p, p', d shape take an
// unrolled path that loads the knots of all five radial functions at once.
// pre() runs once the first knot loads are issued and before the first put2,
// so a caller can wait there for its output buffer while the loads are in flight.
template <bool kNorm = true, typename Put2, typename Pre>
__device__ __forceinline__ bool orbitals_fast2(const SpeciesFast& s, const float2* __restrict__ knot, float ax,
                                               float ay, float az, float bx, float by, float bz, Put2&& put2,
                                               Pre&& pre) {
    const float r2a = ax * ax + ay * ay + az * az;
    const float r2b = bx * bx + by * by + bz * bz;
    const bool ina = r2a < s.rc2, inb = r2b < s.rc2;
    if (!ina && !inb) return false;
    // a point outside the cutoff is evaluated at a safe radius and multiplied by 0
    const float ra = sqrtf(fminf(r2a, s.rc2 * 0.999f)), rb = sqrtf(fminf(r2b, s.rc2 * 0.999f));
    const bool tinya = r2a < 1e-20f, tinyb = r2b < 1e-20f;
    const float ia = tinya ? 0.f : 1.f / ra, ib = tinyb ? 0.f : 1.f / rb;
    const float ma = ina ? 1.f : 0.f, mb = inb ? 1.f : 0.f;
    const float xa = ra * s.inv_dr, xb = rb * s.inv_dr;
    const int ka = min((int)xa, s.n_int - 1), kb = min((int)xb, s.n_int - 1);
    const float ta = xa - (float)ka, tb = xb - (float)kb;
    const float sa = 1.f - ta, qa2 = ta * ta, sb = 1.f - tb, qb2 = tb * tb;
    const float a00 = (1.f + 2.f * ta) * sa * sa, a10 = ta * sa * sa, a01 = qa2 * (3.f - 2.f * ta), a11 = qa2 * (ta - 1.f);
    const float b00 = (1.f + 2.f * tb) * sb * sb, b10 = tb * sb * sb, b01 = qb2 * (3.f - 2.f * tb), b11 = qb2 * (tb - 1.f);
    const int nr = s.n_radial;
    const float2* kna = knot + s.knot2 + ka * nr;
    const float2* knb = knot + s.knot2 + kb * nr;
    // radial part of function j at both points from its knots (p, q: knots k, k + 1), divided by r^l
    auto radial = [&](int l, float2 pa, float2 qa, float2 pb, float2 qb, float& ua, float& ub) {
        ua = (pa.x * a00 + qa.x * a01 + pa.y * a10 + qa.y * a11) * ma;
        ub = (pb.x * b00 + qb.x * b01 + pb.y * b10 + qb.y * b11) * mb;
        if (tinya) ua = (l == 0) ? ua : 0.f;  // centre limit: phi = R(0) Y00 for l = 0, 0 otherwise
        if (tinyb) ub = (l == 0) ? ub : 0.f;
        for (int q = 0; q < l; ++q) { ua *= ia; ub *= ib; }
    };
    if (s.dzp) {
        float2 pa[5], qa[5], pb[5], qb[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            pa[j] = ld_knot(kna + j); qa[j] = ld_knot(kna + 5 + j);
            pb[j] = ld_knot(knb + j); qb[j] = ld_knot(knb + 5 + j);
        }
        pre();  // the knot loads are in flight
        float ua, ub;
        radial(0, pa[0], qa[0], pb[0], qb[0], ua, ub);
        put_l2<0, kNorm>(0, ua, ub, ax, ay, az, bx, by, bz, put2);
        radial(0, pa[1], qa[1], pb[1], qb[1], ua, ub);
        put_l2<0, kNorm>(1, ua, ub, ax, ay, az, bx, by, bz, put2);
        radial(1, pa[2], qa[2], pb[2], qb[2], ua, ub);
        put_l2<1, kNorm>(2, ua, ub, ax, ay, az, bx, by, bz, put2);
        radial(1, pa[3], qa[3], pb[3], qb[3], ua, ub);
        put_l2<1, kNorm>(5, ua, ub, ax, ay, az, bx, by, bz, put2);
        radial(2, pa[4], qa[4], pb[4], qb[4], ua, ub);
        put_l2<2, kNorm>(8, ua, ub, ax, ay, az, bx, by, bz, put2);
        return true;
    }
    // the knots of radial function j + 1 are loaded before the values of j are formed and
    // stored, so their latency overlaps that work
    float2 pa = make_float2(0.f, 0.f), qa = pa, pb = pa, qb = pa;
    if (nr > 0) { pa = ld_knot(kna); qa = ld_knot(kna + nr); pb = ld_knot(knb); qb = ld_knot(knb + nr); }
    pre();
    for (int j = 0; j < nr; ++j) {
        float2 pa1 = pa, qa1 = qa, pb1 = pb, qb1 = qb;
        if (j + 1 < nr) {
            pa1 = ld_knot(kna + j + 1); qa1 = ld_knot(kna + nr + j + 1);
            pb1 = ld_knot(knb + j + 1); qb1 = ld_knot(knb + nr + j + 1);
        }
        const int l = s.rad_l[j];
        const int o = s.orb_base[j];
        float ua, ub;
        radial(l, pa, qa, pb, qb, ua, ub);
        if (l == 0) put_l2<0, kNorm>(o, ua, ub, ax, ay, az, bx, by, bz, put2);
        else if (l == 1) put_l2<1, kNorm>(o, ua, ub, ax, ay, az, bx, by, bz, put2);
        else if (l == 2) put_l2<2, kNorm>(o, ua, ub, ax, ay, az, bx, by, bz, put2);
        else put_l2<3, kNorm>(o, ua, ub, ax, ay, az, bx, by, bz, put2);
        pa = pa1; qa = qa1; pb = pb1; qb = qb1;
    }
    return true;
}
template <bool kNorm = true, typename Put2>
__device__ __forceinline__ bool orbitals_fast2(const SpeciesFast& s, const float2* __restrict__ knot, float ax,
                                               float ay, float az, float bx, float by, float bz, Put2&& put2) {
    return orbitals_fast2<kNorm>(s, knot, ax, ay, az, bx, by, bz, put2, [] {});
}

}  // namespace gint
