// Floating-point operations of one Kalman step of the CUDA path (csrc/kf.cuh), counted exactly by
// instantiating the templates with a scalar type that counts every +, -, *, /, sqrt and asin.
// A fused multiply-add is counted as two operations (it is a multiply and an add).  Prints, per
// hit: the forward step of the gradient kernel (propagation + Joseph update), its adjoint
// (step_bwd, which replays the forward pieces it needs), and the square-root forward step of the
// tracking refit.
#include <cmath>
#include <cstdio>

namespace cnt {
struct Ops {
    long long add = 0, mul = 0, div = 0, sqrt = 0, asin = 0;
};
Ops g_ops;

struct CF {
    double v = 0;
    CF() = default;
    CF(double x) : v(x) {}
    explicit operator int() const { return (int)v; }
};
inline CF operator+(CF a, CF b) { g_ops.add++; return CF(a.v + b.v); }
inline CF operator-(CF a, CF b) { g_ops.add++; return CF(a.v - b.v); }
inline CF operator-(CF a) { return CF(-a.v); }
inline CF operator*(CF a, CF b) { g_ops.mul++; return CF(a.v * b.v); }
inline CF operator/(CF a, CF b) { g_ops.div++; return CF(a.v / b.v); }
inline CF &operator+=(CF &a, CF b) { a = a + b; return a; }
inline CF &operator-=(CF &a, CF b) { a = a - b; return a; }
inline CF &operator*=(CF &a, CF b) { a = a * b; return a; }
inline bool operator<(CF a, CF b) { return a.v < b.v; }
inline bool operator>(CF a, CF b) { return a.v > b.v; }
inline bool operator<=(CF a, CF b) { return a.v <= b.v; }
inline bool operator>=(CF a, CF b) { return a.v >= b.v; }
inline bool operator==(CF a, CF b) { return a.v == b.v; }
inline bool operator!=(CF a, CF b) { return a.v != b.v; }
inline CF k_sqrt(CF a) { g_ops.sqrt++; return CF(std::sqrt(a.v)); }
inline CF k_asin(CF a) { g_ops.asin++; return CF(std::asin(a.v)); }
inline CF k_abs(CF a) { return CF(std::fabs(a.v)); }
inline CF k_fma(CF a, CF b, CF c) { g_ops.mul++; g_ops.add++; return CF(a.v * b.v + c.v); }
}  // namespace cnt

#include "kf.cuh"

using cnt::CF;
using namespace kf;

static long long total(const cnt::Ops &o) { return o.add + o.mul + o.div + o.sqrt + o.asin; }

int main() {
    static CF rc[37], rs[37], xr[159];
    for (int m = -18; m <= 18; m++) {
        rc[m + 18] = CF(std::cos(m * 20 * M_PI / 180));
        rs[m + 18] = CF(std::sin(m * 20 * M_PI / 180));
    }
    for (int r = 0; r < 159; r++) xr[r] = CF(85 + r * 162.0 / 158);
    Geo<CF> g;
    g.kB = CF(-0.299792458e-2 * 0.5);
    g.sig2 = CF(0.01);
    g.smax = CF(0.999);
    g.cmin = CF(0.01);
    g.pitch = CF(162.0 / 158);
    g.half = 18;
    g.rot_c = rc;
    g.rot_s = rs;
    g.xr = xr;
    // a typical state a few rows before a hit of the same sector
    State<CF> s;
    s.x = CF(0.01);
    s.p[0] = CF(0.2); s.p[1] = CF(0.3); s.p[2] = CF(0.2); s.p[3] = CF(0.5); s.p[4] = CF(0.8);
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) s.P[i][j] = CF(i == j ? 0.01 : 0.001);
    s.frame = 3; s.rref = 40; s.yref = CF(1.0); s.zref = CF(50.0);
    FHit<CF> h;
    h.k = 3; h.r = 41; h.xl = CF(0.002); h.yn = CF(1.2); h.yc = CF(0.001); h.zn = CF(50.5); h.zc = CF(0.002);
    h.vy = CF(0.01); h.vz = CF(0.01);

    cnt::g_ops = cnt::Ops();
    State<CF> f = s;
    CF chi2(0);
    step_fwd(f, h, g, chi2);
    const cnt::Ops fwd = cnt::g_ops;

    cnt::g_ops = cnt::Ops();
    Adj<CF> a;
    adj_zero(a);
    for (int i = 0; i < 5; i++) a.p[i] = CF(0.1 * (i + 1));
    CF xb(0), yb(0), zb(0), vyb(0), vzb(0);
    step_bwd(s, h, g, a, &xb, &yb, &zb, &vyb, &vzb);
    const cnt::Ops bwd = cnt::g_ops;

    SqrtState<CF> q;
    q.x = s.x;
    for (int i = 0; i < 5; i++) {
        q.p[i] = s.p[i];
        for (int j = 0; j < 5; j++) q.S[i][j] = CF(i == j ? 0.1 : 0.0);
    }
    q.frame = s.frame; q.rref = s.rref; q.yref = s.yref; q.zref = s.zref;
    cnt::g_ops = cnt::Ops();
    CF chi2q(0);
    sqrt_step(q, h, g, chi2q);
    const cnt::Ops sq = cnt::g_ops;

    std::printf("forward %lld (add %lld mul %lld div %lld sqrt %lld asin %lld)\n", total(fwd), fwd.add, fwd.mul,
                fwd.div, fwd.sqrt, fwd.asin);
    std::printf("adjoint %lld (add %lld mul %lld div %lld sqrt %lld asin %lld)\n", total(bwd), bwd.add, bwd.mul,
                bwd.div, bwd.sqrt, bwd.asin);
    std::printf("sqrt_forward %lld (add %lld mul %lld div %lld sqrt %lld asin %lld)\n", total(sq), sq.add, sq.mul,
                sq.div, sq.sqrt, sq.asin);
    return 0;
}
