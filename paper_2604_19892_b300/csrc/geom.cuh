// Device geometry in FP64: primitive distances, the coplanarity cubic and
// the bisection-based conservative step (supplement Sec. 3).
#pragma once
#include <cuda_runtime.h>

namespace ipcb {

struct d3 {
    double x, y, z;
};
__device__ __forceinline__ d3 mk(double a, double b, double c) { return {a, b, c}; }
__device__ __forceinline__ d3 ld3(const double* p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ d3 operator*(double s, d3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 cross(d3 a, d3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double clamp01(double t) { return fmin(fmax(t, 0.0), 1.0); }

// Closest point of triangle (a, b, c) to p by Voronoi regions; returns the
// squared distance and barycentric weights w of the closest point.
__device__ inline double pt_closest(d3 p, d3 a, d3 b, d3 c, double w[3]) {
    d3 ab = b - a, ac = c - a, ap = p - a;
    double d1 = dot(ab, ap), d2 = dot(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) {
        w[0] = 1; w[1] = 0; w[2] = 0;
        return dot(ap, ap);
    }
    d3 bp = p - b;
    double d3v = dot(ab, bp), d4 = dot(ac, bp);
    if (d3v >= 0.0 && d4 <= d3v) {
        w[0] = 0; w[1] = 1; w[2] = 0;
        return dot(bp, bp);
    }
    double vc = d1 * d4 - d3v * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3v <= 0.0) {
        double t = d1 / (d1 - d3v);
        w[0] = 1 - t; w[1] = t; w[2] = 0;
        d3 q = a + t * ab;
        d3 r = p - q;
        return dot(r, r);
    }
    d3 cp = p - c;
    double d5 = dot(ab, cp), d6 = dot(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) {
        w[0] = 0; w[1] = 0; w[2] = 1;
        return dot(cp, cp);
    }
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        double t = d2 / (d2 - d6);
        w[0] = 1 - t; w[1] = 0; w[2] = t;
        d3 q = a + t * ac;
        d3 r = p - q;
        return dot(r, r);
    }
    double va = d3v * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3v) >= 0.0 && (d5 - d6) >= 0.0) {
        double t = (d4 - d3v) / ((d4 - d3v) + (d5 - d6));
        w[0] = 0; w[1] = 1 - t; w[2] = t;
        d3 q = b + t * (c - b);
        d3 r = p - q;
        return dot(r, r);
    }
    double den = 1.0 / (va + vb + vc);
    double v = vb * den, ww = vc * den;
    w[0] = 1 - v - ww; w[1] = v; w[2] = ww;
    d3 q = a + v * ab + ww * ac;
    d3 r = p - q;
    return dot(r, r);
}

// Closest points of segments p1-q1 and p2-q2 by successive clamping; returns
// the squared distance and the parameters (s, t).
__device__ inline double ee_closest(d3 p1, d3 q1, d3 p2, d3 q2, double& s, double& t) {
    d3 d1 = q1 - p1, d2 = q2 - p2, r = p1 - p2;
    double a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
    const double tiny = 1e-300;
    if (a <= tiny && e <= tiny) {
        s = t = 0.0;
    } else if (a <= tiny) {
        s = 0.0;
        t = clamp01(f / e);
    } else {
        double c = dot(d1, r);
        if (e <= tiny) {
            t = 0.0;
            s = clamp01(-c / a);
        } else {
            double b = dot(d1, d2);
            double den = a * e - b * b;
            s = den > 0.0 ? clamp01((b * f - c * e) / den) : 0.0;
            t = (b * s + f) / e;
            if (t < 0.0) {
                t = 0.0;
                s = clamp01(-c / a);
            } else if (t > 1.0) {
                t = 1.0;
                s = clamp01((b - c) / a);
            }
        }
    }
    d3 c1 = p1 + s * d1, c2 = p2 + t * d2;
    d3 dd = c1 - c2;
    return dot(dd, dd);
}

// ---- FP32 prefilter: a conservative lower bound on a pair's distance.
// Positions enter as FP64 differences from the pair's first vertex (so large
// coordinates keep their relative accuracy), the closest-point computation
// runs in FP32, and the bound subtracts a margin far above FP32 rounding.
struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 fsub(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ float fdot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 fmad3(f3 a, float t, f3 b) { return {a.x + t * b.x, a.y + t * b.y, a.z + t * b.z}; }
__device__ __forceinline__ float fclamp01(float t) { return fminf(fmaxf(t, 0.f), 1.f); }

// Squared point-triangle distance by the Voronoi regions of the triangle
// (vertices, edges, face), the published closest-point method of C. Ericson,
// Real-Time Collision Detection (2005), Sec. 5.1.5.
__device__ inline float pt_dist2_f(f3 p, f3 a, f3 b, f3 c) {
    f3 ab = fsub(b, a), ac = fsub(c, a), ap = fsub(p, a);
    float d1 = fdot(ab, ap), d2 = fdot(ac, ap);
    if (d1 <= 0.f && d2 <= 0.f) return fdot(ap, ap);
    f3 bp = fsub(p, b);
    float d3v = fdot(ab, bp), d4 = fdot(ac, bp);
    if (d3v >= 0.f && d4 <= d3v) return fdot(bp, bp);
    float vc = d1 * d4 - d3v * d2;
    if (vc <= 0.f && d1 >= 0.f && d3v <= 0.f) {
        f3 r = fsub(p, fmad3(a, d1 / (d1 - d3v), ab));
        return fdot(r, r);
    }
    f3 cp = fsub(p, c);
    float d5 = fdot(ab, cp), d6 = fdot(ac, cp);
    if (d6 >= 0.f && d5 <= d6) return fdot(cp, cp);
    float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
        f3 r = fsub(p, fmad3(a, d2 / (d2 - d6), ac));
        return fdot(r, r);
    }
    float va = d3v * d6 - d5 * d4;
    if (va <= 0.f && (d4 - d3v) >= 0.f && (d5 - d6) >= 0.f) {
        f3 r = fsub(p, fmad3(b, (d4 - d3v) / ((d4 - d3v) + (d5 - d6)), fsub(c, b)));
        return fdot(r, r);
    }
    float den = 1.f / (va + vb + vc);
    f3 q = fmad3(fmad3(a, vb * den, ab), vc * den, ac);
    f3 r = fsub(p, q);
    return fdot(r, r);
}

// Squared segment-segment distance: the unconstrained line parameters clamped
// to [0, 1], the other parameter recomputed and clamped in turn (Ericson,
// Real-Time Collision Detection (2005), Sec. 5.1.9).
__device__ inline float ee_dist2_f(f3 p1, f3 q1, f3 p2, f3 q2) {
    f3 d1 = fsub(q1, p1), d2 = fsub(q2, p2), r = fsub(p1, p2);
    float a = fdot(d1, d1), e = fdot(d2, d2), f = fdot(d2, r);
    float s, t;
    const float tiny = 1e-30f;
    if (a <= tiny && e <= tiny) {
        s = t = 0.f;
    } else if (a <= tiny) {
        s = 0.f;
        t = fclamp01(f / e);
    } else {
        float c = fdot(d1, r);
        if (e <= tiny) {
            t = 0.f;
            s = fclamp01(-c / a);
        } else {
            float b = fdot(d1, d2);
            float den = a * e - b * b;
            s = den > 0.f ? fclamp01((b * f - c * e) / den) : 0.f;
            t = (b * s + f) / e;
            if (t < 0.f) {
                t = 0.f;
                s = fclamp01(-c / a);
            } else if (t > 1.f) {
                t = 1.f;
                s = fclamp01((b - c) / a);
            }
        }
    }
    f3 dd = fsub(fmad3(p1, s, d1), fmad3(p2, t, d2));
    return fdot(dd, dd);
}

// f(t) = det[A + t dA, B + t dB, C + t dC] = c[0] + c[1] t + c[2] t^2 + c[3] t^3
__device__ inline void cubic_of(d3 A, d3 dA, d3 B, d3 dB, d3 C, d3 dC, double c[4]) {
    d3 BC = cross(B, C);
    d3 mid = cross(dB, C) + cross(B, dC);
    d3 dBdC = cross(dB, dC);
    c[0] = dot(A, BC);
    c[1] = dot(dA, BC) + dot(A, mid);
    c[2] = dot(dA, mid) + dot(A, dBdC);
    c[3] = dot(dA, dBdC);
}

__device__ __forceinline__ double horner(const double c[4], double t) { return ((c[3] * t + c[2]) * t + c[1]) * t + c[0]; }
__device__ __forceinline__ int sgn(double v) { return (v > 0.0) - (v < 0.0); }

// 16 fixed halvings keeping the safe end (supplement Algorithm 1).
__device__ inline double safe_bisect(const double c[4], double xs, double xu, double ys) {
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
        double xm = 0.5 * (xs + xu);
        double ym = horner(c, xm);
        if (sgn(ym) != sgn(ys)) {
            xu = xm;
        } else {
            xs = xm;
            ys = ym;
        }
    }
    return xs;
}

// Largest safe step in [alpha_l, 1] by walking the monotone pieces of f
// (supplement Algorithm 2).
__device__ inline double cubic_safe(const double c[4], double al) {
    if (al >= 1.0) return 1.0;
    double x = fmax(al, 0.0);
    const double x0 = x;
    double y = horner(c, x);
    if (y == 0.0) return x;
    double e[3];
    int n = 0;
    double A = c[3], B = c[2], Cc = c[1];
    double disc = B * B - 3.0 * A * Cc;
    if (disc > 0.0) {
        double q = -(B + copysign(sqrt(disc), B >= 0.0 ? 1.0 : -1.0));
        double r1 = q / (3.0 * A), r2 = Cc / q;
        double lo = fmin(r1, r2), hi = fmax(r1, r2);
        if (lo > x && lo < 1.0) e[n++] = lo;
        if (hi > x && hi < 1.0 && hi > lo) e[n++] = hi;
    } else if (disc == 0.0 && A != 0.0) {
        double ti = -B / (3.0 * A);
        if (ti > x && ti < 1.0) e[n++] = ti;
    }
    e[n++] = 1.0;
    for (int i = 0; i < n; ++i) {
        double ye = horner(c, e[i]);
        if (sgn(ye) != sgn(y)) return x > x0 ? x : safe_bisect(c, x, e[i], y);
        x = e[i];
        y = ye;
    }
    return 1.0;
}

}  // namespace ipcb
