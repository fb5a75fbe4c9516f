// Host check of the hand-written Kalman-filter adjoints of the CUDA path (csrc/kf.cuh), compiled in
// double precision with the host compiler: every backward function is compared with central
// differences of its forward function.  The objective is chi2 plus a fixed linear functional of
// the final state and covariance, so that every adjoint path (state, covariance, chi2) is live.
// Sequence (the step from the first hit to the vertex and the reference updates):
//   prop_fwd(dx, dyref, dzref) -> upd_fwd_joseph(y, z) -> upd1_fwd(z) -> upd1_fwd(tan lambda)
//   -> upd1_fwd(q/pT)
// and, separately, one rotation into the neighbouring sector followed by a propagation and a
// two-coordinate update with unequal variances (also checking the measurement and variance
// adjoints).  Prints the largest relative error and exits 0.
#include <cmath>
#include <cstdio>
#include <random>

#include "kf.cuh"

using namespace kf;
typedef double T;

static const T KB = -0.299792458e-2 * 0.5;

struct Lin {          // objective weights on the final state
    T w[5];
    T W[5][5];
};

static T objective(const State<T> &s, const Lin &L, T chi2) {
    T f = chi2;
    for (int i = 0; i < 5; i++) {
        f += L.w[i] * s.p[i];
        for (int j = 0; j < 5; j++) f += L.W[i][j] * s.P[i][j];
    }
    return f;
}

struct Meas {
    T dx, dy, dz, s2v, mz, Rz, mt, Rt, mq, Rq;
};

static T run_anchor(State<T> s, T dx, const Meas &m, const Lin &L, bool *ok) {
    *ok = prop_fwd(s, dx, KB, T(0.999), m.dy, m.dz);
    if (!*ok) return 0;
    T chi2 = upd_fwd_joseph(s, T(0), T(0), m.s2v, m.s2v);
    chi2 += upd1_fwd(s, 1, m.mz, m.Rz);
    chi2 += upd1_fwd(s, 3, m.mt, m.Rt);
    chi2 += upd1_fwd(s, 4, m.mq, m.Rq);
    return objective(s, L, chi2);
}

static T run_rot(State<T> s, T ca, T sa, T dx, T ym, T zm, T vy, T vz, const Lin &L, bool *ok) {
    *ok = rot_fwd(s, ca, sa, KB, T(0.01));
    if (!*ok) return 0;
    *ok = prop_fwd(s, dx, KB, T(0.999));
    if (!*ok) return 0;
    const T chi2 = upd_fwd_joseph(s, ym, zm, vy, vz);
    return objective(s, L, chi2);
}

static void random_state(std::mt19937 &rng, State<T> &s) {
    std::uniform_real_distribution<T> U(-1, 1);
    s.x = 3.0 * U(rng);
    s.p[0] = 2.0 * U(rng);
    s.p[1] = 5.0 * U(rng);
    s.p[2] = 0.4 * U(rng);
    s.p[3] = 0.8 * U(rng);
    s.p[4] = 0.3 + 2.0 * std::fabs(U(rng));
    if (U(rng) < 0) s.p[4] = -s.p[4];
    T A[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) A[i][j] = U(rng) * (i == j ? 1.0 : 0.3);
    const T sc[5] = {0.05, 0.05, 1e-3, 1e-3, 1e-2};
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            T v = 0;
            for (int k = 0; k < 5; k++) v += A[i][k] * A[j][k];
            s.P[i][j] = v * sc[i] * sc[j] + (i == j ? 0.1 * sc[i] * sc[i] : 0.0);
        }
    s.frame = 0;
    s.rref = 0;
    s.yref = s.zref = 0;
}

static void random_lin(std::mt19937 &rng, Lin &L) {
    std::uniform_real_distribution<T> U(-1, 1);
    for (int i = 0; i < 5; i++) {
        L.w[i] = U(rng);
        for (int j = 0; j <= i; j++) L.W[i][j] = L.W[j][i] = 100.0 * U(rng);
    }
}

static T relerr(T fd, T an, T scale) { return std::fabs(fd - an) / (std::fabs(fd) + scale); }

// Largest |fd - adjoint| over the state entries, and separately over the covariance entries, each
// relative to the largest |fd| of its group.
template <class F>
static T check_inputs(State<T> s, const Adj<T> &a, F f) {
    T dp = 0, mp = 0, dP = 0, mP = 0;
    for (int i = 0; i < 5; i++) {
        const T e = 1e-6 * (std::fabs(s.p[i]) + 1e-2);
        State<T> sp = s, sm = s;
        sp.p[i] += e;
        sm.p[i] -= e;
        bool o1, o2;
        const T fd = (f(sp, &o1) - f(sm, &o2)) / (2 * e);
        dp = std::fmax(dp, std::fabs(fd - a.p[i]));
        mp = std::fmax(mp, std::fabs(fd));
    }
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) {
            const T e = 1e-6 * std::sqrt(s.P[i][i] * s.P[j][j]);
            State<T> sp = s, sm = s;
            sp.P[i][j] += e;
            sm.P[i][j] -= e;
            if (i != j) {
                sp.P[j][i] += e;
                sm.P[j][i] -= e;
            }
            bool o1, o2;
            const T fd = (f(sp, &o1) - f(sm, &o2)) / (2 * e);
            const T an = i == j ? a.G[i][j] : a.G[i][j] + a.G[j][i];
            // compare on the scale of the perturbation: d f for a one-sigma-relative change
            const T sc = std::sqrt(s.P[i][i] * s.P[j][j]);
            dP = std::fmax(dP, std::fabs(fd - an) * sc);
            mP = std::fmax(mP, std::fabs(fd) * sc);
        }
    return std::fmax(dp / (mp + 1e-300), dP / (mP + 1e-300));
}

int main() {
    std::mt19937 rng(7);
    std::normal_distribution<T> N(0, 1);
    T worst = 0;
    int n = 0;
    for (int trial = 0; trial < 200; trial++) {
        State<T> s;
        random_state(rng, s);
        Lin L;
        random_lin(rng, L);
        const T dx = -(80.0 + 100.0 * std::fabs(N(rng)) * 0.3);
        // forward to the vertex plane (y, z near 0 after the reference shift)
        State<T> t = s;
        if (!prop_fwd(t, dx, KB, T(0.999))) continue;
        Meas m;
        m.dx = dx;
        m.dy = t.p[0] + 0.01 * N(rng);
        m.dz = t.p[1] + 0.01 * N(rng);
        m.s2v = 1e-4;
        m.mz = 0.01 * N(rng);
        m.Rz = 1e-4;
        m.mt = s.p[3] + 1e-3 * N(rng);
        m.Rt = 1e-6;
        m.mq = s.p[4] * (1 + 0.01 * N(rng));
        m.Rq = 1e-4 * s.p[4] * s.p[4];
        bool ok;
        const T f0 = run_anchor(s, dx, m, L, &ok);
        if (!ok) continue;
        // adjoint: stage inputs
        State<T> s0 = s, s1 = s;
        prop_fwd(s1, dx, KB, T(0.999), m.dy, m.dz);
        State<T> s2 = s1;
        upd_fwd_joseph(s2, T(0), T(0), m.s2v, m.s2v);
        State<T> s3 = s2;
        upd1_fwd(s3, 1, m.mz, m.Rz);
        State<T> s4 = s3;
        upd1_fwd(s4, 3, m.mt, m.Rt);
        Adj<T> a;
        adj_zero(a);
        for (int i = 0; i < 5; i++) {
            a.p[i] = L.w[i];
            for (int j = 0; j < 5; j++) a.G[i][j] = L.W[i][j];
        }
        upd1_bwd(s4, 4, m.mq, m.Rq, a);
        upd1_bwd(s3, 3, m.mt, m.Rt, a);
        upd1_bwd(s2, 1, m.mz, m.Rz, a);
        T ymb, zmb, vyb, vzb;
        upd_bwd(s1, T(0), T(0), m.s2v, m.s2v, a, &ymb, &zmb, &vyb, &vzb);
        const T dxb = prop_bwd(s0, dx, KB, T(0.999), a);
        const T scale = 1e-3 * (std::fabs(f0) + 1.0);
        worst = std::fmax(worst, check_inputs(s, a, [&](const State<T> &v, bool *o) {
            return run_anchor(v, dx, m, L, o); }));
        {
            const T e = 1e-6 * std::fabs(dx);
            bool o1, o2;
            const T fd = (run_anchor(s, dx + e, m, L, &o1) - run_anchor(s, dx - e, m, L, &o2)) / (2 * e);
            worst = std::fmax(worst, relerr(fd, dxb, scale));
        }
        // rotation + propagation + update
        const T da = (trial % 2 ? 1.0 : -1.0) * 20.0 * M_PI / 180.0;
        const T ca = std::cos(da), sa = std::sin(da);
        State<T> r = s;
        r.x = 100.0 + s.x;
        const T dx2 = 1.3 + 0.2 * N(rng);
        State<T> rr = r;
        if (!rot_fwd(rr, ca, sa, KB, T(0.01))) continue;
        State<T> rp = rr;
        if (!prop_fwd(rp, dx2, KB, T(0.999))) continue;
        const T ym = rp.p[0] + 0.1 * N(rng), zm = rp.p[1] + 0.1 * N(rng);
        const T vy = 0.01 * (1 + 0.3 * std::fabs(N(rng))), vz = 0.01 * (1 + 0.3 * std::fabs(N(rng)));
        Adj<T> b;
        adj_zero(b);
        for (int i = 0; i < 5; i++) {
            b.p[i] = L.w[i];
            for (int j = 0; j < 5; j++) b.G[i][j] = L.W[i][j];
        }
        upd_bwd(rp, ym, zm, vy, vz, b, &ymb, &zmb, &vyb, &vzb);
        prop_bwd(rr, dx2, KB, T(0.999), b);
        rot_bwd(r, ca, sa, KB, b);
        {   // measurement and variance adjoints
            const T ev = 1e-6;
            bool o1, o2;
            const T f1 = run_rot(r, ca, sa, dx2, ym, zm, vy, vz, L, &ok);
            const T sc = 1e-6 * (std::fabs(f1) + 1.0);
            T fd = (run_rot(r, ca, sa, dx2, ym + ev, zm, vy, vz, L, &o1) -
                    run_rot(r, ca, sa, dx2, ym - ev, zm, vy, vz, L, &o2)) / (2 * ev);
            worst = std::fmax(worst, relerr(fd, ymb, sc));
            fd = (run_rot(r, ca, sa, dx2, ym, zm + ev, vy, vz, L, &o1) -
                  run_rot(r, ca, sa, dx2, ym, zm - ev, vy, vz, L, &o2)) / (2 * ev);
            worst = std::fmax(worst, relerr(fd, zmb, sc));
            const T eV = 1e-7;
            fd = (run_rot(r, ca, sa, dx2, ym, zm, vy + eV, vz, L, &o1) -
                  run_rot(r, ca, sa, dx2, ym, zm, vy - eV, vz, L, &o2)) / (2 * eV);
            worst = std::fmax(worst, relerr(fd, vyb, sc / 0.01));
            fd = (run_rot(r, ca, sa, dx2, ym, zm, vy, vz + eV, L, &o1) -
                  run_rot(r, ca, sa, dx2, ym, zm, vy, vz - eV, L, &o2)) / (2 * eV);
            worst = std::fmax(worst, relerr(fd, vzb, sc / 0.01));
        }
        worst = std::fmax(worst, check_inputs(r, b, [&](const State<T> &v, bool *o) {
            return run_rot(v, ca, sa, dx2, ym, zm, vy, vz, L, o); }));
        n++;
    }
    std::printf("cases %d worst_rel_err %.3e\n", n, worst);
    return 0;
}
