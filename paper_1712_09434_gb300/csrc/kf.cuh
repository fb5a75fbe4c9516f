// Kalman-filter helix refit and its hand-written adjoint (arxiv 1712.09434 section 3: Kalman
// filter track fitting; the final track refit of the merger).  Header-only, templated on the
// scalar type; the library instantiates it in float.
//
// State (y, z, sin phi, tan lambda, q/pT) at local x in the frame of the current hit's sector;
// covariance P (symmetric 5x5, kept as a full matrix in registers).  One step =
//   rotation into the hit's sector if it changed (reference surface moved with the point),
//   exact helix propagation to the hit's x (C = kB q/pT; sin phi2 = sin phi + C dx;
//     dy = dx T, T = (sin phi + sin phi2)/(cos phi + cos phi2); L = dx sqrt(1+T^2);
//     dz = tan lambda * L * asin(C L/2)/(C L/2)), covariance F P F^T with the step Jacobian,
//   measurement update with (y, z), R = diag(vy, vz), symmetric form P - U S^-1 U^T.
//
// The adjoint propagates d(sum chi2)/d(.) backwards through one step.  Matrix adjoints use the
// symmetric-gradient convention: for a symmetric argument P, Pb is symmetric and
// d f = sum_ij Pb_ij dP_ij.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define KF_HD __host__ __device__ __forceinline__
#else
#define KF_HD inline
#endif

namespace kf {

KF_HD float k_sqrt(float a) { return sqrtf(a); }
KF_HD double k_sqrt(double a) { return sqrt(a); }
KF_HD float k_asin(float a) { return asinf(a); }
KF_HD double k_asin(double a) { return asin(a); }
KF_HD float k_abs(float a) { return fabsf(a); }
KF_HD double k_abs(double a) { return fabs(a); }
KF_HD float k_fma(float a, float b, float c) { return fmaf(a, b, c); }
KF_HD double k_fma(double a, double b, double c) { return fma(a, b, c); }

// asin(u)/u and its derivative; power series for small |u| (coefficients of the Taylor series of
// asin(u)/u = sum (2k)!/(4^k (k!)^2 (2k+1)) u^(2k)).
template <class T>
KF_HD T asinc(T u) {
    const T u2 = u * u;
    if (k_abs(u) < T(0.25))
        return T(1) + u2 * (T(1.0 / 6) + u2 * (T(3.0 / 40) + u2 * (T(5.0 / 112) + u2 * (T(35.0 / 1152) +
               u2 * (T(63.0 / 2816) + u2 * T(231.0 / 13312))))));
    return k_asin(u) / u;
}
template <class T>
KF_HD T asinc_d(T u) {
    const T u2 = u * u;
    if (k_abs(u) < T(0.25))
        return u * (T(2.0 / 6) + u2 * (T(12.0 / 40) + u2 * (T(30.0 / 112) + u2 * (T(8 * 35.0 / 1152) +
               u2 * (T(10 * 63.0 / 2816) + u2 * T(12 * 231.0 / 13312))))));
    return (u / k_sqrt(T(1) - u2) - k_asin(u)) / u2;
}

// Positions are kept relative to the nominal coordinates of a reference hit (the last hit
// processed): absolute x = xr[rref] + x, y = yref + p[0], z = zref + p[1].  Nominal coordinates
// are exact in FP32 (row planes, multiples of the fixed-point unit), so the state carries only
// small offsets of the size of a residual and the FP32 rounding of absolute coordinates up to
// 250 cm never enters the filter.  The references are calibration-independent constants: they
// move the origin, not the function, so derivatives are unchanged.
template <class T>
struct State {
    T x;
    T p[5];
    T P[5][5];
    int frame;
    int rref;
    T yref, zref;
};

template <class T>
struct Adj {
    T x;
    T p[5];
    T G[5][5];
};

template <class T>
KF_HD void adj_zero(Adj<T> &a) {
    a.x = T(0);
    for (int i = 0; i < 5; i++) {
        a.p[i] = T(0);
        for (int j = 0; j < 5; j++) a.G[i][j] = T(0);
    }
}

// ---- sector rotation --------------------------------------------------------------------------
// Rotate by da (cos ca, sin sa) into the new frame.  Returns false if cos phi' <= cmin.
template <class T>
KF_HD bool rot_fwd(State<T> &s, T ca, T sa, T kB, T cmin) {
    const T sn = s.p[2];
    const T cs = k_sqrt(T(1) - sn * sn);
    const T x1 = s.x * ca + s.p[0] * sa;
    const T y1 = -s.x * sa + s.p[0] * ca;
    const T sn1 = sn * ca - cs * sa;
    const T cs1 = cs * ca + sn * sa;
    if (!(cs1 > cmin)) return false;
    const T C = kB * s.p[4];
    const T j00 = cs / cs1, j10 = -s.p[3] * sa / cs1, j20 = -C * sa, j22 = cs1 / cs;
    // P <- J P J^T, J = I except rows 0,1,2 / column 0 and (2,2)
    T A[5][5];
    for (int j = 0; j < 5; j++) {
        A[0][j] = j00 * s.P[0][j];
        A[1][j] = j10 * s.P[0][j] + s.P[1][j];
        A[2][j] = j20 * s.P[0][j] + j22 * s.P[2][j];
        A[3][j] = s.P[3][j];
        A[4][j] = s.P[4][j];
    }
    // P' = A J^T, symmetric: the lower triangle, mirrored
    auto col = [&](int i, int j) -> T {
        switch (j) {
            case 0: return j00 * A[i][0];
            case 1: return j10 * A[i][0] + A[i][1];
            case 2: return j20 * A[i][0] + j22 * A[i][2];
            default: return A[i][j];
        }
    };
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) {
            const T v = col(i, j);
            s.P[i][j] = v;
            s.P[j][i] = v;
        }
    s.x = x1;
    s.p[0] = y1;
    s.p[2] = sn1;
    return true;
}

// Adjoint of rot_fwd.  `s` is the state BEFORE the rotation; a holds the adjoint of the state
// after it and is overwritten with the adjoint of the state before it.
template <class T>
KF_HD void rot_bwd(const State<T> &s, T ca, T sa, T kB, Adj<T> &a) {
    const T sn = s.p[2], tl = s.p[3], q = s.p[4];
    const T cs = k_sqrt(T(1) - sn * sn);
    const T cs1 = cs * ca + sn * sa;
    const T ic1 = T(1) / cs1;
    const T C = kB * q;
    const T j00 = cs * ic1, j10 = -tl * sa * ic1, j20 = -C * sa, j22 = cs1 / cs;
    // Jb = 2 G' J P at the state-dependent entries (0,0), (1,0), (2,0), (2,2)
    T GJ[5][5];   // G' J
    for (int i = 0; i < 5; i++) {
        GJ[i][0] = a.G[i][0] * j00 + a.G[i][1] * j10 + a.G[i][2] * j20;
        GJ[i][1] = a.G[i][1];
        GJ[i][2] = a.G[i][2] * j22;
        GJ[i][3] = a.G[i][3];
        GJ[i][4] = a.G[i][4];
    }
    T Jb00 = T(0), Jb10 = T(0), Jb20 = T(0), Jb22 = T(0);
    for (int k = 0; k < 5; k++) {
        Jb00 += GJ[0][k] * s.P[k][0];
        Jb10 += GJ[1][k] * s.P[k][0];
        Jb20 += GJ[2][k] * s.P[k][0];
        Jb22 += GJ[2][k] * s.P[k][2];
    }
    Jb00 *= T(2);
    Jb10 *= T(2);
    Jb20 *= T(2);
    Jb22 *= T(2);
    // G <- J^T G' J (symmetric: the lower triangle, mirrored)
    auto row = [&](int i, int j) -> T {
        switch (i) {
            case 0: return j00 * GJ[0][j] + j10 * GJ[1][j] + j20 * GJ[2][j];
            case 2: return j22 * GJ[2][j];
            default: return GJ[i][j];
        }
    };
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) {
            const T v = row(i, j);
            a.G[i][j] = v;
            a.G[j][i] = v;
        }
    // state: x1 = x ca + y sa, y1 = -x sa + y ca, sn1 = sn ca - cs sa, (z, tl, q) unchanged,
    // plus the Jacobian entries' dependence on (sn, tl, q).
    T xb = a.x * ca - a.p[0] * sa;
    T yb = a.x * sa + a.p[0] * ca;
    T snb = a.p[2] * ca;
    T csb = -a.p[2] * sa;
    T tlb = a.p[3];
    T qb = a.p[4];
    T zb = a.p[1];
    // j00 = cs ic1 ; j10 = -tl sa ic1 ; j20 = -C sa ; j22 = cs1 / cs
    T ic1b = Jb00 * cs - Jb10 * tl * sa;
    csb += Jb00 * ic1 - Jb22 * cs1 / (cs * cs);
    tlb += -Jb10 * sa * ic1;
    T Cb = -Jb20 * sa;
    T cs1b = Jb22 / cs - ic1b * ic1 * ic1;
    // cs1 = cs ca + sn sa
    csb += cs1b * ca;
    snb += cs1b * sa;
    // cs = sqrt(1 - sn^2)
    snb += -csb * sn / cs;
    qb += Cb * kB;
    a.x = xb;
    a.p[0] = yb;
    a.p[1] = zb;
    a.p[2] = snb;
    a.p[3] = tlb;
    a.p[4] = qb;
}

// ---- helix propagation ------------------------------------------------------------------------
template <class T>
struct PropV {   // forward intermediates of one propagation step
    T dx, C, s2, c1, c2, ic1, ic2, den, T_, W, sW, L, u, f, arc, h, g2;
    T F02, F04, F12, F13, F14, F24;
};

template <class T, class St>
KF_HD bool prop_vals(const St &s, T dx, T kB, T smax, PropV<T> &v) {
    const T sn = s.p[2], tl = s.p[3], q = s.p[4];
    v.dx = dx;
    v.C = kB * q;
    v.s2 = sn + v.C * v.dx;
    if (!(k_abs(v.s2) < smax) || !(k_abs(sn) < smax)) return false;
    v.c1 = k_sqrt(T(1) - sn * sn);
    v.c2 = k_sqrt(T(1) - v.s2 * v.s2);
    v.ic1 = T(1) / v.c1;
    v.ic2 = T(1) / v.c2;
    v.den = v.c1 + v.c2;
    v.T_ = (sn + v.s2) / v.den;
    v.W = T(1) + v.T_ * v.T_;
    v.sW = k_sqrt(v.W);
    v.L = v.dx * v.sW;
    v.u = T(0.5) * v.C * v.L;
    v.f = asinc(v.u);
    v.arc = v.L * v.f;
    v.h = T(0.5) * (v.ic1 + v.ic2);
    v.g2 = T(0.5) * v.ic2 * kB * v.dx * v.dx;
    v.F02 = v.dx * v.W * v.h;
    v.F04 = v.W * v.g2;
    v.F12 = tl * v.dx * v.T_ * v.sW * v.h;
    v.F13 = v.arc;
    v.F14 = tl * v.T_ * v.sW * v.g2;
    v.F24 = kB * v.dx;
    return true;
}

// Propagate by dx along the helix and move the (y, z) origin by (dyref, dzref) (the caller updates
// the reference x).
template <class T>
KF_HD bool prop_fwd(State<T> &s, T dx, T kB, T smax, T dyref = T(0), T dzref = T(0)) {
    PropV<T> v;
    if (!prop_vals(s, dx, kB, smax, v)) return false;
    const T a = v.F02, b = v.F04, c = v.F12, d = v.F13, e = v.F14, f = v.F24;
    T A[5][5];
    for (int j = 0; j < 5; j++) {
        A[0][j] = s.P[0][j] + a * s.P[2][j] + b * s.P[4][j];
        A[1][j] = s.P[1][j] + c * s.P[2][j] + d * s.P[3][j] + e * s.P[4][j];
        A[2][j] = s.P[2][j] + f * s.P[4][j];
        A[3][j] = s.P[3][j];
        A[4][j] = s.P[4][j];
    }
    // P' = A F^T, symmetric: the lower triangle, mirrored
    auto col = [&](int i, int j) -> T {
        switch (j) {
            case 0: return A[i][0] + a * A[i][2] + b * A[i][4];
            case 1: return A[i][1] + c * A[i][2] + d * A[i][3] + e * A[i][4];
            case 2: return A[i][2] + f * A[i][4];
            default: return A[i][j];
        }
    };
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) {
            const T v = col(i, j);
            s.P[i][j] = v;
            s.P[j][i] = v;
        }
    s.p[0] += v.dx * v.T_ - dyref;
    s.p[1] += s.p[3] * v.arc - dzref;
    s.p[2] = v.s2;
    return true;
}

// Adjoint of prop_fwd; `s` is the state before the step.  Returns the adjoint of dx (a.x, the
// adjoint of the reference x, is left to the caller).
template <class T>
KF_HD T prop_bwd(const State<T> &s, T dx, T kB, T smax, Adj<T> &a) {
    PropV<T> v;
    prop_vals(s, dx, kB, smax, v);
    const T sn = s.p[2], tl = s.p[3];
    // F = I + F02 e0e2' + F04 e0e4' + F12 e1e2' + F13 e1e3' + F14 e1e4' + F24 e2e4'; products
    // written out over its non-zero entries.  GF = G' F:
    T GF[5][5];
    for (int i = 0; i < 5; i++) {
        GF[i][0] = a.G[i][0];
        GF[i][1] = a.G[i][1];
        GF[i][2] = a.G[i][2] + a.G[i][0] * v.F02 + a.G[i][1] * v.F12;
        GF[i][3] = a.G[i][3] + a.G[i][1] * v.F13;
        GF[i][4] = a.G[i][4] + a.G[i][0] * v.F04 + a.G[i][1] * v.F14 + a.G[i][2] * v.F24;
    }
    // Fb = 2 G' F P at the six state-dependent entries
    T F02b = T(0), F04b = T(0), F12b = T(0), F13b = T(0), F14b = T(0), F24b = T(0);
    for (int k = 0; k < 5; k++) {
        F02b += GF[0][k] * s.P[k][2];
        F04b += GF[0][k] * s.P[k][4];
        F12b += GF[1][k] * s.P[k][2];
        F13b += GF[1][k] * s.P[k][3];
        F14b += GF[1][k] * s.P[k][4];
        F24b += GF[2][k] * s.P[k][4];
    }
    F02b *= T(2); F04b *= T(2); F12b *= T(2); F13b *= T(2); F14b *= T(2); F24b *= T(2);
    // G <- F^T G' F = F^T GF (symmetric: the lower triangle, mirrored)
    auto row = [&](int i, int j) -> T {
        switch (i) {
            case 2: return GF[2][j] + v.F02 * GF[0][j] + v.F12 * GF[1][j];
            case 3: return GF[3][j] + v.F13 * GF[1][j];
            case 4: return GF[4][j] + v.F04 * GF[0][j] + v.F14 * GF[1][j] + v.F24 * GF[2][j];
            default: return GF[i][j];
        }
    };
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) {
            const T g = row(i, j);
            a.G[i][j] = g;
            a.G[j][i] = g;
        }

    // state outputs: y' = y + dx T, z' = z + tl arc, s' = s2, tl' = tl, q' = q, x' = xh
    const T ypb = a.p[0], zpb = a.p[1], spb = a.p[2];
    T yb = ypb, zb = zpb, tlb = a.p[3], qb = a.p[4];
    T dxb = T(0), Tb = T(0), arcb = T(0), s2b = spb, snb = T(0);
    // Jacobian entries
    arcb += F13b;
    // F14 = tl T sW g2
    tlb += F14b * v.T_ * v.sW * v.g2;
    Tb += F14b * tl * v.sW * v.g2;
    T sWb = F14b * tl * v.T_ * v.g2;
    T g2b = F14b * tl * v.T_ * v.sW;
    // F12 = tl dx T sW h
    tlb += F12b * v.dx * v.T_ * v.sW * v.h;
    dxb += F12b * tl * v.T_ * v.sW * v.h;
    Tb += F12b * tl * v.dx * v.sW * v.h;
    sWb += F12b * tl * v.dx * v.T_ * v.h;
    T hb = F12b * tl * v.dx * v.T_ * v.sW;
    // F04 = W g2
    T Wb = F04b * v.g2;
    g2b += F04b * v.W;
    // F02 = dx W h
    dxb += F02b * v.W * v.h;
    Wb += F02b * v.dx * v.h;
    hb += F02b * v.dx * v.W;
    // F24 = kB dx
    dxb += F24b * kB;
    // g2 = 0.5 ic2 kB dx^2
    T ic2b = g2b * T(0.5) * kB * v.dx * v.dx;
    dxb += g2b * v.ic2 * kB * v.dx;
    // h = 0.5 (ic1 + ic2)
    T ic1b = T(0.5) * hb;
    ic2b += T(0.5) * hb;
    // state part
    T dyb = ypb;                 // y' = y + dy, dy = dx T
    tlb += zpb * v.arc;          // z' = z + tl arc
    arcb += zpb * tl;
    // arc = L f
    T Lb = arcb * v.f;
    T fb = arcb * v.L;
    // f = asinc(u)
    T ub = fb * asinc_d(v.u);
    // u = 0.5 C L
    T Cb = ub * T(0.5) * v.L;
    Lb += ub * T(0.5) * v.C;
    // L = dx sW
    dxb += Lb * v.sW;
    sWb += Lb * v.dx;
    // sW = sqrt(W)
    Wb += sWb * T(0.5) / v.sW;
    // W = 1 + T^2
    Tb += Wb * T(2) * v.T_;
    // dy = dx T
    dxb += dyb * v.T_;
    Tb += dyb * v.dx;
    // T = (sn + s2) / den
    const T numb = Tb / v.den;
    const T denb = -Tb * v.T_ / v.den;
    snb += numb;
    s2b += numb;
    T c1b = denb, c2b = denb;
    // ic = 1/c
    c1b += -ic1b * v.ic1 * v.ic1;
    c2b += -ic2b * v.ic2 * v.ic2;
    // c = sqrt(1 - s^2)
    snb += -c1b * sn * v.ic1;
    s2b += -c2b * v.s2 * v.ic2;
    // s2 = sn + C dx
    snb += s2b;
    Cb += s2b * v.dx;
    dxb += s2b * v.C;
    // C = kB q
    qb += Cb * kB;
    a.p[0] = yb;
    a.p[1] = zb;
    a.p[2] = snb;
    a.p[3] = tlb;
    a.p[4] = qb;
    return dxb;
}

// ---- measurement update ----------------------------------------------------------------------
template <class T>
KF_HD T upd_fwd(State<T> &s, T ym, T zm, T vy, T vz) {
    const T r0 = ym - s.p[0], r1 = zm - s.p[1];
    const T S00 = s.P[0][0] + vy, S01 = s.P[0][1], S11 = s.P[1][1] + vz;
    const T idet = T(1) / (S00 * S11 - S01 * S01);
    const T i00 = S11 * idet, i01 = -S01 * idet, i11 = S00 * idet;
    const T chi2 = r0 * r0 * i00 + T(2) * r0 * r1 * i01 + r1 * r1 * i11;
    T U0[5], U1[5], K0[5], K1[5];
    for (int j = 0; j < 5; j++) {
        U0[j] = s.P[j][0];
        U1[j] = s.P[j][1];
        K0[j] = U0[j] * i00 + U1[j] * i01;
        K1[j] = U0[j] * i01 + U1[j] * i11;
    }
    for (int j = 0; j < 5; j++) s.p[j] += K0[j] * r0 + K1[j] * r1;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) {
            const T v = s.P[i][j] - (K0[i] * U0[j] + K1[i] * U1[j]);
            s.P[i][j] = v;
            s.P[j][i] = v;
        }
    return chi2;
}

// Adjoint of upd_fwd with d(chi2) = 1; `s` is the state before the update.  Writes the adjoint
// of the measurement to (*ymb, *zmb) and that of the variances (vy, vz) to (*vyb, *vzb).
template <class T>
KF_HD void upd_bwd(const State<T> &s, T ym, T zm, T vy, T vz, Adj<T> &a, T *ymb, T *zmb, T *vyb, T *vzb) {
    const T r0 = ym - s.p[0], r1 = zm - s.p[1];
    const T S00 = s.P[0][0] + vy, S01 = s.P[0][1], S11 = s.P[1][1] + vz;
    const T idet = T(1) / (S00 * S11 - S01 * S01);
    const T i00 = S11 * idet, i01 = -S01 * idet, i11 = S00 * idet;
    // U = P H^T (columns 0, 1 of P), K = U Si.  With pb the adjoint of p' = p + K r and w = U^T pb:
    // K^T pb = Si w, and Kb = pb r^T is rank one.
    T U[5][2];
    T w0 = T(0), w1 = T(0);
#pragma unroll
    for (int j = 0; j < 5; j++) {
        U[j][0] = s.P[j][0];
        U[j][1] = s.P[j][1];
        w0 += U[j][0] * a.p[j];
        w1 += U[j][1] * a.p[j];
    }
    // rb = K^T pb + 2 Si r = Si (w + 2 r)
    const T e0 = w0 + T(2) * r0, e1 = w1 + T(2) * r1;
    const T rb0 = i00 * e0 + i01 * e1, rb1 = i01 * e0 + i11 * e1;
    // GU = G'' U  (5x2)
    T GU[5][2];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        T g0 = T(0), g1 = T(0);
#pragma unroll
        for (int k = 0; k < 5; k++) {
            g0 += a.G[i][k] * U[k][0];
            g1 += a.G[i][k] * U[k][1];
        }
        GU[i][0] = g0;
        GU[i][1] = g1;
    }
    // M = U^T G'' U (symmetric)
    T M00 = T(0), M01 = T(0), M11 = T(0);
#pragma unroll
    for (int k = 0; k < 5; k++) {
        M00 += U[k][0] * GU[k][0];
        M01 += U[k][0] * GU[k][1];
        M11 += U[k][1] * GU[k][1];
    }
    // Sib = r r^T - M + U^T Kb = r r^T - M + w r^T, symmetrised
    const T sb00 = r0 * r0 - M00 + w0 * r0;
    const T sb11 = r1 * r1 - M11 + w1 * r1;
    const T sb01 = r0 * r1 - M01 + T(0.5) * (w0 * r1 + w1 * r0);
    // Ub = (-2 G'' U + Kb) Si = -2 GU Si + pb (Si r)^T
    const T q0 = i00 * r0 + i01 * r1, q1 = i01 * r0 + i11 * r1;
    T Ub[5][2];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        Ub[j][0] = T(-2) * (GU[j][0] * i00 + GU[j][1] * i01) + a.p[j] * q0;
        Ub[j][1] = T(-2) * (GU[j][0] * i01 + GU[j][1] * i11) + a.p[j] * q1;
    }
    // Sb = -Si Sib Si
    const T t00 = i00 * sb00 + i01 * sb01, t01 = i00 * sb01 + i01 * sb11;
    const T t10 = i01 * sb00 + i11 * sb01, t11 = i01 * sb01 + i11 * sb11;
    const T Sb00 = -(t00 * i00 + t01 * i01), Sb01 = -(t00 * i01 + t01 * i11);
    const T Sb11 = -(t10 * i01 + t11 * i11);
    // G' = G'' + sym(G_U) + Sb on the (0:2, 0:2) block
#pragma unroll
    for (int j = 0; j < 5; j++) {
        a.G[j][0] += T(0.5) * Ub[j][0];
        a.G[0][j] += T(0.5) * Ub[j][0];
        a.G[j][1] += T(0.5) * Ub[j][1];
        a.G[1][j] += T(0.5) * Ub[j][1];
    }
    a.G[0][0] += Sb00;
    a.G[0][1] += Sb01;
    a.G[1][0] += Sb01;
    a.G[1][1] += Sb11;
    // p' adjoint
    a.p[0] -= rb0;
    a.p[1] -= rb1;
    *ymb = rb0;
    *zmb = rb1;
    *vyb = Sb00;              // S = P_mm + R
    *vzb = Sb11;
}

}  // namespace kf

namespace kf {

// Per-call constants of the fit.
template <class T>
struct Geo {
    T kB, sig2, smax, cmin, pitch;
    int half;               // sectors per side
    const T *rot_c;         // cos(m * sector width), index m + half, m in [-half, half]
    const T *rot_s;
    const T *xr;            // row plane radii
};

// Rotation index between frames: the sector-angle difference wrapped into (-180, 180] degrees.
KF_HD int rot_index(int k_new, int k_old, int half) {
    int m = (k_new % half) - (k_old % half);
    if (2 * m > half) m -= half;
    if (2 * m <= -half) m += half;
    return m + half;
}

// A hit as the filter sees it: sector kh, row rh, nominal (yn, zn) and the calibration offsets
// (xl, yc, zc): x = xr[rh] + xl, y = yn + yc, z = zn + zc; measurement variances (vy, vz).
template <class T>
struct FHit {
    int k, r;
    T xl, yn, yc, zn, zc, vy, vz;
};

// Rotation into the frame of the hit's sector (absolute coordinates), re-referenced to the hit.
template <class T>
KF_HD bool step_rotate(State<T> &s, const FHit<T> &h, const Geo<T> &g) {
    const int m = rot_index(h.k, s.frame, g.half);
    s.x = g.xr[s.rref] + s.x;
    s.p[0] = s.yref + s.p[0];
    if (!rot_fwd(s, g.rot_c[m], g.rot_s[m], g.kB, g.cmin)) return false;
    s.x = s.x - g.xr[h.r];
    s.p[0] = s.p[0] - h.yn;
    s.p[1] = s.p[1] + (s.zref - h.zn);
    s.rref = h.r;
    s.yref = h.yn;
    s.zref = h.zn;
    s.frame = h.k;
    return true;
}

// One Kalman step to hit h.  Returns false if the track leaves the domain of the local
// parametrisation (then the fit fails).
template <class T>
KF_HD bool step_fwd(State<T> &s, const FHit<T> &h, const Geo<T> &g, T &chi2) {
    if (h.k != s.frame && !step_rotate(s, h, g)) return false;
    const T dx = T(h.r - s.rref) * g.pitch + (h.xl - s.x);
    if (!prop_fwd(s, dx, g.kB, g.smax, h.yn - s.yref, h.zn - s.zref)) return false;
    s.x = h.xl;
    s.rref = h.r;
    s.yref = h.yn;
    s.zref = h.zn;
    chi2 += upd_fwd_joseph(s, h.yc, h.zc, h.vy, h.vz);
    return true;
}

// Adjoint of step_fwd (for a step that succeeded): `s_in` is the state before the step, `a` the
// adjoint after it (overwritten with the adjoint before it); adds the adjoints of the hit's
// calibration offsets (xl, yc, zc) to *xb, *yb, *zb and those of its variances to *vyb, *vzb.
template <class T>
KF_HD void step_bwd(const State<T> &s_in, const FHit<T> &h, const Geo<T> &g, Adj<T> &a, T *xb, T *yb, T *zb,
                    T *vyb, T *vzb) {
    State<T> s1 = s_in;
    const bool rot = h.k != s_in.frame;
    if (rot) step_rotate(s1, h, g);
    const T dx = T(h.r - s1.rref) * g.pitch + (h.xl - s1.x);
    State<T> s2 = s1;
    prop_fwd(s2, dx, g.kB, g.smax, h.yn - s1.yref, h.zn - s1.zref);
    s2.x = h.xl;
    s2.rref = h.r;
    s2.yref = h.yn;
    s2.zref = h.zn;
    T ymb, zmb, vyb_, vzb_;
    upd_bwd(s2, h.yc, h.zc, h.vy, h.vz, a, &ymb, &zmb, &vyb_, &vzb_);
    *yb += ymb;
    *zb += zmb;
    *vyb += vyb_;
    *vzb += vzb_;
    const T dxb = prop_bwd(s1, dx, g.kB, g.smax, a);
    *xb += a.x + dxb;         // xl is both the new reference offset and part of dx
    a.x = -dxb;               // the old offset enters only through dx
    if (rot) {                // absolute x1, y1 = rotation; s1 offsets = absolute - constants
        const int m = rot_index(h.k, s_in.frame, g.half);
        rot_bwd(s_in, g.rot_c[m], g.rot_s[m], g.kB, a);
    }
}

// Seed at the last hit E from the circle through A (first), B (middle) and E, all already in E's
// frame: signed curvature from the three points, direction at E = chord A->E plus half the
// turning angle, tan lambda = dz / arc.  Returns false for a degenerate triple.
template <class T>
KF_HD bool seed3(T ax, T ay, T az, T bx, T by, T ex, T ey, T ez, T kB, T smax, T p[5]) {
    const T abx = bx - ax, aby = by - ay, bex = ex - bx, bey = ey - by, aex = ex - ax, aey = ey - ay;
    const T lab = k_sqrt(abx * abx + aby * aby), lbe = k_sqrt(bex * bex + bey * bey);
    const T lae = k_sqrt(aex * aex + aey * aey);
    if (!(lab > T(0)) || !(lbe > T(0)) || !(lae > T(0))) return false;
    // cross product ab x be by Kahan's fused-multiply-add determinant: for a nearly straight
    // track the two products cancel to the sagitta, which this keeps to about one ulp
    const T w = aby * bex;
    const T cross = k_fma(abx, bey, -w) + k_fma(-aby, bex, w);
    const T kappa = T(2) * cross / (lab * lbe * lae);
    const T u = T(0.5) * kappa * lae;
    if (!(k_abs(u) < T(1))) return false;
    // sin(atan2(aey, aex) + asin(u)) = (aey cos(asin u) + aex u) / lae
    const T cu = k_sqrt(T(1) - u * u);
    const T sn = (aey * cu + aex * u) / lae;
    if (!(k_abs(sn) < smax)) return false;
    p[0] = ey;
    p[1] = ez;
    p[2] = sn;
    p[3] = (ez - az) / (lae * asinc(u));
    p[4] = kappa / kB;
    return true;
}

}  // namespace kf

namespace kf {

// Measurement update in Joseph form: P <- A P A^T + K R K^T with A = I - K H.  The measured 2x2
// block of A is R S^-1 (= I - P_mm S^-1, computed without cancellation), the other rows are -K.
// Algebraically equal to upd_fwd (same state, same chi2, same covariance for the optimal gain);
// numerically it keeps the covariance positive and avoids the large-minus-large cancellation of
// P - U S^-1 U^T when a loose prior meets the first measurements.
template <class T>
KF_HD T upd_fwd_joseph(State<T> &s, T ym, T zm, T vy, T vz) {
    const T r0 = ym - s.p[0], r1 = zm - s.p[1];
    const T S00 = s.P[0][0] + vy, S01 = s.P[0][1], S11 = s.P[1][1] + vz;
    const T idet = T(1) / (S00 * S11 - S01 * S01);
    const T i00 = S11 * idet, i01 = -S01 * idet, i11 = S00 * idet;
    const T chi2 = r0 * r0 * i00 + T(2) * r0 * r1 * i01 + r1 * r1 * i11;
    T K[5][2];
    for (int j = 0; j < 5; j++) {
        K[j][0] = s.P[j][0] * i00 + s.P[j][1] * i01;
        K[j][1] = s.P[j][0] * i01 + s.P[j][1] * i11;
    }
    // A columns 0,1 (A = I - K H): rows 0,1 = R S^-1, rows 2..4 = -K
    T A[5][2];
    A[0][0] = vy * i00; A[0][1] = vy * i01;
    A[1][0] = vz * i01; A[1][1] = vz * i11;
    for (int j = 2; j < 5; j++) { A[j][0] = -K[j][0]; A[j][1] = -K[j][1]; }
    // B = A P (A = [A_c | e_2 e_3 e_4 columns]): B_ij = A_i0 P_0j + A_i1 P_1j + [i>=2] P_ij; the lower
    // triangle of P_new = B A^T + K R K^T needs columns 0, 1 of B and its lower part from column 2
    auto B = [&](int i, int j) { return A[i][0] * s.P[0][j] + A[i][1] * s.P[1][j] + (i >= 2 ? s.P[i][j] : T(0)); };
    T B0[5], B1[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        B0[i] = B(i, 0);
        B1[i] = B(i, 1);
    }
    T Pn[5][5];
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++)
            Pn[i][j] = B0[i] * A[j][0] + B1[i] * A[j][1] + (j >= 2 ? B(i, j) : T(0)) + vy * K[i][0] * K[j][0] +
                       vz * K[i][1] * K[j][1];
    for (int j = 0; j < 5; j++) s.p[j] += K[j][0] * r0 + K[j][1] * r1;
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) {
            s.P[i][j] = Pn[i][j];
            s.P[j][i] = Pn[i][j];
        }
    return chi2;
}

}  // namespace kf

namespace kf {

// Scalar measurement m of state component i with variance R (plain symmetric form):
// u = P e_i, S = P_ii + R, r = m - p_i; p <- p + u r/S, P <- P - u u^T/S, chi2 += r^2/S.
template <class T>
KF_HD T upd1_fwd(State<T> &s, int i, T m, T R) {
    T u[5];
    for (int j = 0; j < 5; j++) u[j] = s.P[j][i];
    const T S = u[i] + R;
    const T iS = T(1) / S;
    const T r = m - s.p[i];
    const T g = r * iS;
    for (int j = 0; j < 5; j++) s.p[j] += u[j] * g;
    for (int a = 0; a < 5; a++)
        for (int b = 0; b <= a; b++) {
            const T v = s.P[a][b] - u[a] * u[b] * iS;
            s.P[a][b] = v;
            s.P[b][a] = v;
        }
    return r * g;
}

// Adjoint of upd1_fwd with d(chi2) = 1; `s` is the state before the update, `a` the adjoint after
// it (overwritten with the adjoint before it).  The measured value is a constant.
template <class T>
KF_HD void upd1_bwd(const State<T> &s, int i, T m, T R, Adj<T> &a) {
    T u[5];
    for (int j = 0; j < 5; j++) u[j] = s.P[j][i];
    const T S = u[i] + R;
    const T iS = T(1) / S;
    const T r = m - s.p[i];
    const T g = r * iS;
    // p' = p + u g ; chi2 = r g ; P' = P - u u^T / S
    T gb = T(0), uGu = T(0);
    T Gu[5];
    for (int j = 0; j < 5; j++) {
        gb += a.p[j] * u[j];
        T acc = T(0);
        for (int k = 0; k < 5; k++) acc += a.G[j][k] * u[k];
        Gu[j] = acc;
        uGu += u[j] * acc;
    }
    T ub[5];
    for (int j = 0; j < 5; j++) ub[j] = a.p[j] * g - T(2) * Gu[j] * iS;
    const T rb = gb * iS + T(2) * g;                 // from g = r/S and chi2 = r^2/S
    const T Sb = -gb * g * iS - g * g + uGu * iS * iS;   // d/dS of g = r/S, chi2 = r^2/S, u u^T/S
    // u = P e_i (symmetric split), S = P_ii + R, r = m - p_i
    for (int j = 0; j < 5; j++) {
        a.G[j][i] += T(0.5) * ub[j];
        a.G[i][j] += T(0.5) * ub[j];
    }
    a.G[i][i] += Sb;
    a.p[i] -= rb;
}

}  // namespace kf

namespace kf {

// ---- square-root form of the forward filter ----------------------------------------------------
// The same filter with the covariance carried as a square root, P = S S^T (S a general 5x5
// matrix).  A linear map J acts as S <- J S; a scalar measurement of component i with variance R
// is Potter's square-root update: phi = S^T e_i, a = 1/(phi.phi + R), g = 1/(1 + sqrt(a R)),
// K = a S phi, S <- S - g a (S phi) phi^T, which is P <- P - K e_i^T P exactly.  The (y, z)
// measurement with diagonal R is processed as two scalar updates (the same posterior and the same
// total chi2 as the joint update).  In FP32 the square root halves the digits the covariance loses
// to its condition number.
template <class T>
struct SqrtState {
    T x;
    T p[5];
    T S[5][5];
    int frame;
    int rref;
    T yref, zref;
};

template <class T>
KF_HD bool sqrt_rot(SqrtState<T> &s, T ca, T sa, T kB, T cmin) {
    const T sn = s.p[2];
    const T cs = k_sqrt(T(1) - sn * sn);
    const T x1 = s.x * ca + s.p[0] * sa;
    const T y1 = -s.x * sa + s.p[0] * ca;
    const T sn1 = sn * ca - cs * sa;
    const T cs1 = cs * ca + sn * sa;
    if (!(cs1 > cmin)) return false;
    const T C = kB * s.p[4];
    const T j00 = cs / cs1, j10 = -s.p[3] * sa / cs1, j20 = -C * sa, j22 = cs1 / cs;
    for (int j = 0; j < 5; j++) {
        const T s0 = s.S[0][j];
        s.S[0][j] = j00 * s0;
        s.S[1][j] = j10 * s0 + s.S[1][j];
        s.S[2][j] = j20 * s0 + j22 * s.S[2][j];
    }
    s.x = x1;
    s.p[0] = y1;
    s.p[2] = sn1;
    return true;
}

template <class T>
KF_HD bool sqrt_prop(SqrtState<T> &s, T dx, T kB, T smax, T dyref, T dzref) {
    PropV<T> v;
    if (!prop_vals(s, dx, kB, smax, v)) return false;
    for (int j = 0; j < 5; j++) {
        const T s2 = s.S[2][j], s3 = s.S[3][j], s4 = s.S[4][j];
        s.S[0][j] += v.F02 * s2 + v.F04 * s4;
        s.S[1][j] += v.F12 * s2 + v.F13 * s3 + v.F14 * s4;
        s.S[2][j] += v.F24 * s4;
    }
    s.p[0] += v.dx * v.T_ - dyref;
    s.p[1] += s.p[3] * v.arc - dzref;
    s.p[2] = v.s2;
    return true;
}

template <class T>
KF_HD T sqrt_upd1(SqrtState<T> &s, int i, T m, T R) {
    T phi[5], Sphi[5];
    T pp = T(0);
    for (int j = 0; j < 5; j++) {
        phi[j] = s.S[i][j];
        pp += phi[j] * phi[j];
    }
    for (int a = 0; a < 5; a++) {
        T v = T(0);
        for (int j = 0; j < 5; j++) v += s.S[a][j] * phi[j];
        Sphi[a] = v;
    }
    const T alpha = T(1) / (pp + R);
    const T gamma = T(1) / (T(1) + k_sqrt(alpha * R));
    const T r = m - s.p[i];
    const T ar = alpha * r, ga = gamma * alpha;
    for (int a = 0; a < 5; a++) {
        s.p[a] += Sphi[a] * ar;
        for (int b = 0; b < 5; b++) s.S[a][b] -= ga * Sphi[a] * phi[b];
    }
    return r * ar;
}

// One step to hit h in square-root form (same geometry as step_fwd).
template <class T>
KF_HD bool sqrt_step(SqrtState<T> &s, const FHit<T> &h, const Geo<T> &g, T &chi2) {
    if (h.k != s.frame) {
        const int m = rot_index(h.k, s.frame, g.half);
        s.x = g.xr[s.rref] + s.x;
        s.p[0] = s.yref + s.p[0];
        if (!sqrt_rot(s, g.rot_c[m], g.rot_s[m], g.kB, g.cmin)) return false;
        s.x = s.x - g.xr[h.r];
        s.p[0] = s.p[0] - h.yn;
        s.p[1] = s.p[1] + (s.zref - h.zn);
        s.rref = h.r;
        s.yref = h.yn;
        s.zref = h.zn;
        s.frame = h.k;
    }
    const T dx = T(h.r - s.rref) * g.pitch + (h.xl - s.x);
    if (!sqrt_prop(s, dx, g.kB, g.smax, h.yn - s.yref, h.zn - s.zref)) return false;
    s.x = h.xl;
    s.rref = h.r;
    s.yref = h.yn;
    s.zref = h.zn;
    chi2 += sqrt_upd1(s, 0, h.yc, h.vy);
    chi2 += sqrt_upd1(s, 1, h.zc, h.vz);
    return true;
}

}  // namespace kf
