// Host-side FP64 construction of velocity sets (Sec. 3.2) and meshes (Sec. 3.1).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sllbm_internal.h"

namespace sllbm {

namespace {

const double kPhi = 0.5 * (1.0 + std::sqrt(5.0));
const double kPi = 3.14159265358979323846;

void push_shell(std::vector<double>& xi, const std::vector<std::array<double, 3>>& reps, double radius, int D) {
    for (int sgn = 1; sgn >= -1; sgn -= 2)
        for (const auto& r : reps) {
            double n = 0;
            for (int d = 0; d < D; ++d) n += r[d] * r[d];
            n = std::sqrt(n);
            for (int d = 0; d < D; ++d) xi.push_back(sgn * r[d] / n * radius);
        }
}

// cyclic permutations of (0, a, b) in the order (0,a,b), (b,0,a), (a,b,0)
std::array<double, 3> cyc(int k, double a, double b) {
    if (k == 0) return {0.0, a, b};
    if (k == 1) return {b, 0.0, a};
    return {a, b, 0.0};
}

}  // namespace

int build_velocity_set(int kind, HostVelSet& vs, std::string& err) {
    vs.xi.clear();
    vs.w.clear();
    vs.opp.clear();
    vs.shell_s.clear();
    if (kind == SLLBM_D2Q9) {
        vs.Q = 9;
        vs.D = 2;
        const double s = std::sqrt(3.0);
        const double p[9][2] = {{0, 0}, {s, 0}, {0, s}, {s, s}, {-s, s}, {-s, 0}, {0, -s}, {-s, -s}, {s, -s}};
        for (auto& q : p) {
            vs.xi.push_back(q[0]);
            vs.xi.push_back(q[1]);
        }
        vs.w = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36};
        vs.shell_s = {0.0, 3.0, 6.0};
    } else if (kind == SLLBM_D2Q19) {
        vs.Q = 19;
        vs.D = 2;
        const double r15 = std::sqrt(15.0);
        const double ra2 = (48.0 - 8.0 * r15) / 7.0, rc2 = (48.0 + 8.0 * r15) / 7.0;
        const double radii[3] = {std::sqrt(ra2), 2.0 * std::sqrt(2.0), std::sqrt(rc2)};
        const double a0[3] = {0.0, kPi / 6.0, 0.0};
        vs.xi = {0.0, 0.0};
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 6; ++k) {
                const double ang = a0[r] + k * kPi / 3.0;
                vs.xi.push_back(radii[r] * std::cos(ang));
                vs.xi.push_back(radii[r] * std::sin(ang));
            }
        // weights: rest 31/96, middle ring 1/128; the two remaining rings from
        // sum w = 1 and sum w |xi|^2 = D:  6 (wa + wc) = 121/192, 6 (wa ra2 + wc rc2) = 13/8
        const double wb = 1.0 / 128.0;
        const double S0 = 121.0 / 1152.0, S2 = 13.0 / 48.0;
        const double wa = (S2 - rc2 * S0) / (ra2 - rc2);
        const double wc = S0 - wa;
        vs.w.push_back(31.0 / 96.0);
        for (int k = 0; k < 6; ++k) vs.w.push_back(wa);
        for (int k = 0; k < 6; ++k) vs.w.push_back(wb);
        for (int k = 0; k < 6; ++k) vs.w.push_back(wc);
        vs.shell_s = {0.0, ra2, 8.0, rc2};
    } else if (kind == SLLBM_D2Q25) {
        vs.Q = 25;
        vs.D = 2;
        const double r10 = std::sqrt(10.0);
        const double r1 = std::sqrt(5.0 - r10), r2 = std::sqrt(5.0 + r10);
        const double x[5] = {0.0, r1, r2, -r1, -r2};
        const double w1d[5] = {8.0 / 15.0, (7.0 + 2.0 * r10) / 60.0, (7.0 - 2.0 * r10) / 60.0,
                               (7.0 + 2.0 * r10) / 60.0, (7.0 - 2.0 * r10) / 60.0};
        for (int b = 0; b < 5; ++b)
            for (int a = 0; a < 5; ++a) {
                vs.xi.push_back(x[a]);
                vs.xi.push_back(x[b]);
                vs.w.push_back(w1d[a] * w1d[b]);
            }
        const double c[3] = {0.0, r1 * r1, r2 * r2};
        vs.shell_s = {0.0, c[1], c[2], 2 * c[1], c[1] + c[2], 2 * c[2]};
    } else if (kind == SLLBM_D3Q45) {
        vs.Q = 45;
        vs.D = 3;
        vs.xi = {0.0, 0.0, 0.0};
        std::vector<std::array<double, 3>> ico = {cyc(0, kPhi, 1), cyc(0, -kPhi, 1), cyc(1, kPhi, 1),
                                                  cyc(1, -kPhi, 1), cyc(2, kPhi, 1), cyc(2, -kPhi, 1)};
        std::vector<std::array<double, 3>> dod = {{1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {-1, 1, 1},
                                                  cyc(0, 1 / kPhi, kPhi), cyc(0, -1 / kPhi, kPhi),
                                                  cyc(1, 1 / kPhi, kPhi), cyc(1, -1 / kPhi, kPhi),
                                                  cyc(2, 1 / kPhi, kPhi), cyc(2, -1 / kPhi, kPhi)};
        push_shell(vs.xi, ico, std::sqrt(3.0), 3);
        push_shell(vs.xi, dod, 3.0, 3);
        push_shell(vs.xi, ico, std::sqrt(15.0), 3);
        vs.w.push_back(28.0 / 135.0);
        for (int k = 0; k < 12; ++k) vs.w.push_back(25.0 / 432.0);
        for (int k = 0; k < 20; ++k) vs.w.push_back(1.0 / 216.0);
        for (int k = 0; k < 12; ++k) vs.w.push_back(1.0 / 2160.0);
        vs.shell_s = {0.0, 3.0, 9.0, 15.0};
    } else if (kind == SLLBM_D3Q125) {
        // product of the 5-point Gauss-Hermite rule (weight exp(-x^2/2) / sqrt(2 pi)):
        // nodes 0, +-sqrt(5 -+ sqrt10), weights 8/15 and (7 +- 2 sqrt10)/60
        vs.Q = 125;
        vs.D = 3;
        const double r10 = std::sqrt(10.0);
        const double r1 = std::sqrt(5.0 - r10), r2 = std::sqrt(5.0 + r10);
        const double x[5] = {0.0, r1, r2, -r1, -r2};
        const double w1d[5] = {8.0 / 15.0, (7.0 + 2.0 * r10) / 60.0, (7.0 - 2.0 * r10) / 60.0,
                               (7.0 + 2.0 * r10) / 60.0, (7.0 - 2.0 * r10) / 60.0};
        for (int c = 0; c < 5; ++c)
            for (int b = 0; b < 5; ++b)
                for (int a = 0; a < 5; ++a) {
                    vs.xi.push_back(x[a]);
                    vs.xi.push_back(x[b]);
                    vs.xi.push_back(x[c]);
                    vs.w.push_back(w1d[a] * w1d[b] * w1d[c]);
                }
    } else {
        err = "unknown velocity set";
        return SLLBM_ERR_ARG;
    }
    // opposite indices by search (the sets are symmetric under xi -> -xi)
    vs.opp.assign(vs.Q, -1);
    for (int i = 0; i < vs.Q; ++i) {
        double best = 1e300;
        for (int j = 0; j < vs.Q; ++j) {
            double dd = 0;
            for (int d = 0; d < vs.D; ++d) dd += std::fabs(vs.xi[i * vs.D + d] + vs.xi[j * vs.D + d]);
            if (dd < best) {
                best = dd;
                vs.opp[i] = j;
            }
        }
        if (best > 1e-12) {
            err = "velocity set is not symmetric";
            return SLLBM_ERR_ARG;
        }
    }
    return SLLBM_OK;
}

int build_custom_velocity_set(const sllbm_velset_desc& d, HostVelSet& vs, std::string& err) {
    if (d.Q < 1 || d.Q > SLLBM_QMAX_GENERIC || (d.D != 2 && d.D != 3) || !d.xi || !d.w) {
        err = "custom velocity set: 1 <= Q <= " + std::to_string(SLLBM_QMAX_GENERIC) +
              ", D = 2 or 3 and both arrays required";
        return SLLBM_ERR_ARG;
    }
    vs.Q = d.Q;
    vs.D = d.D;
    vs.xi.assign(d.xi, d.xi + size_t(d.Q) * d.D);
    vs.w.assign(d.w, d.w + d.Q);
    vs.opp.assign(d.Q, -1);
    vs.shell_s.clear();
    for (double v : vs.xi)
        if (!std::isfinite(v)) {
            err = "custom velocity set: non-finite abscissa";
            return SLLBM_ERR_ARG;
        }
    for (double v : vs.w)
        if (!std::isfinite(v) || !(v > 0.0)) {
            err = "custom velocity set: weights must be positive and finite";
            return SLLBM_ERR_ARG;
        }
    const int D = d.D;
    for (int i = 0; i < d.Q; ++i) {
        double best = 1e300;
        for (int j = 0; j < d.Q; ++j) {
            double dd = 0;
            for (int a = 0; a < D; ++a) dd += std::fabs(vs.xi[i * D + a] + vs.xi[j * D + a]);
            if (dd < best) {
                best = dd;
                vs.opp[i] = j;
            }
        }
        if (best > 1e-12 || std::fabs(vs.w[vs.opp[i]] - vs.w[i]) > 1e-14 * std::max(1.0, vs.w[i])) {
            err = "custom velocity set: not symmetric under xi -> -xi (with equal weights)";
            return SLLBM_ERR_ARG;
        }
    }
    // moments of the weight function to second order: sum w = 1, sum w xi = 0,
    // sum w xi xi = identity (units of sqrt(T0))
    double m0 = 0, m1[3] = {0, 0, 0}, m2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < d.Q; ++i) {
        m0 += vs.w[i];
        for (int a = 0; a < D; ++a) {
            m1[a] += vs.w[i] * vs.xi[i * D + a];
            for (int b = 0; b < D; ++b) m2[a][b] += vs.w[i] * vs.xi[i * D + a] * vs.xi[i * D + b];
        }
    }
    bool ok = std::fabs(m0 - 1.0) <= 1e-10;
    for (int a = 0; a < D; ++a) {
        ok = ok && std::fabs(m1[a]) <= 1e-10;
        for (int b = 0; b < D; ++b) ok = ok && std::fabs(m2[a][b] - (a == b ? 1.0 : 0.0)) <= 1e-10;
    }
    if (!ok) {
        err = "custom velocity set: moments to second order differ from the weight function's "
              "(sum w = 1, sum w xi = 0, sum w xi xi = I within 1e-10)";
        return SLLBM_ERR_ARG;
    }
    return SLLBM_OK;
}

// ------------------------------------------------------------ meshes
namespace {

double naca_half(double x, double t) {
    x = std::min(1.0, std::max(0.0, x));
    return 5.0 * t * (0.2969 * std::sqrt(x) - 0.1260 * x - 0.3516 * x * x + 0.2843 * x * x * x -
                      0.1036 * x * x * x * x);
}

}  // namespace

int build_mesh(const sllbm_mesh_desc& d, HostMesh& m, std::string& err) {
    m = HostMesh();
    m.kind = d.kind;
    m.D = d.dim;
    m.p = d.p;
    if (d.dim < 2 || d.dim > 3) { err = "dim must be 2 or 3"; return SLLBM_ERR_ARG; }
    if (d.p < 1 || d.p > 4) { err = "p must be in 1..4"; return SLLBM_ERR_ARG; }
    for (int k = 0; k < d.dim; ++k) {
        if (d.cells[k] < 1 || d.cells[k] > (1 << 20)) { err = "bad cell count"; return SLLBM_ERR_ARG; }
        if (!(d.length[k] > 0) && d.kind != SLLBM_MESH_EXPLICIT) { err = "lengths must be positive"; return SLLBM_ERR_ARG; }
        m.cells[k] = d.cells[k];
        m.length[k] = d.length[k];
    }
    m.stretch = d.stretch;
    m.thickness = d.thickness;
    m.central = d.central;
    for (int k = 0; k < 3; ++k) m.periodic[k] = 1;
    if (d.kind == SLLBM_MESH_BOX) {
    } else if (d.kind == SLLBM_MESH_CHANNEL || d.kind == SLLBM_MESH_MIXING) {
        m.periodic[1] = 0;
    } else if (d.kind == SLLBM_MESH_NACA) {
        if (d.dim != 2) { err = "NACA mesh is 2D"; return SLLBM_ERR_ARG; }
        m.periodic[1] = 0;
        if (d.cells[0] < 8 || d.cells[1] < 1) { err = "NACA mesh too small"; return SLLBM_ERR_ARG; }
    } else if (d.kind == SLLBM_MESH_EXPLICIT) {
        const bool p0 = d.bc[0].kind == SLLBM_BC_PERIODIC, p1 = d.bc[1].kind == SLLBM_BC_PERIODIC;
        if (p0 != p1) { err = "explicit mesh: y is periodic at both ends or at neither"; return SLLBM_ERR_ARG; }
        m.periodic[1] = p0 ? 1 : 0;
        for (int k = 0; k < d.dim; ++k) {
            const double* v = d.vertices[k];
            if (!v) { err = "explicit mesh: vertices[" + std::to_string(k) + "] is NULL"; return SLLBM_ERR_ARG; }
            for (int j = 0; j <= d.cells[k]; ++j)
                if (!std::isfinite(v[j]) || (j > 0 && !(v[j] > v[j - 1]))) {
                    err = "explicit mesh: vertices[" + std::to_string(k) + "] must be finite and strictly increasing";
                    return SLLBM_ERR_ARG;
                }
            if (m.periodic[k] && v[0] != 0.0) {
                err = "explicit mesh: a periodic dimension starts at 0 (vertices[" + std::to_string(k) + "][0])";
                return SLLBM_ERR_ARG;
            }
            m.length[k] = v[d.cells[k]] - v[0];
        }
    } else {
        err = "unknown mesh kind";
        return SLLBM_ERR_ARG;
    }
    m.glc.resize(d.p + 1);
    for (int k = 0; k <= d.p; ++k) m.glc[k] = -std::cos(kPi * k / d.p);
    m.n_nodes = 1;
    m.n_cells = 1;
    for (int k = 0; k < d.dim; ++k) {
        m.N[k] = m.periodic[k] ? d.cells[k] * d.p : d.cells[k] * d.p + 1;
        m.n_nodes *= m.N[k];
        m.n_cells *= m.cells[k];
    }
    if (m.n_nodes >= (int64_t(1) << 31)) { err = "too many nodes"; return SLLBM_ERR_ARG; }
    if (m.n_cells >= (int64_t(1) << 24)) { err = "too many cells (limit 2^24)"; return SLLBM_ERR_ARG; }
    const int D = d.dim;
    m.X.assign(size_t(m.n_nodes) * D, 0.0);
    auto node_logical = [&](int dd, int k) {
        int c = std::min(k / d.p, m.cells[dd] - 1);
        int a = k - c * d.p;
        return std::make_pair(c, 0.5 * (m.glc[a] + 1.0));
    };
    if (d.kind != SLLBM_MESH_NACA) {
        for (int dd = 0; dd < D; ++dd) {
            const int C = m.cells[dd];
            const double L = m.length[dd];
            auto& V = m.V[dd];
            V.resize(C + 1);
            if (d.kind == SLLBM_MESH_EXPLICIT) {
                V.assign(d.vertices[dd], d.vertices[dd] + C + 1);
                if (m.periodic[dd])
                    for (int j = 0; j < C; ++j)
                        if (std::fabs((V[j + 1] - V[j]) - L / C) > 1e-12 * L) m.uniform_periodic = false;
            } else if (dd != 1 || d.kind == SLLBM_MESH_BOX) {
                for (int j = 0; j <= C; ++j) V[j] = L * j / C;
            } else if (d.kind == SLLBM_MESH_CHANNEL) {
                const double b = d.stretch;
                if (!(b > 0)) { err = "channel stretch must be > 0"; return SLLBM_ERR_ARG; }
                for (int j = 0; j <= C; ++j)
                    V[j] = 0.5 * L * (1.0 - std::tanh(b * (1.0 - 2.0 * j / C)) / std::tanh(b));
            } else {
                const int nc = d.central;
                const int side = (C - nc) / 2;
                if (nc < 1 || 2 * side + nc != C || !(d.stretch >= 1.0)) {
                    err = "mixing mesh: central cells must leave an even remainder; stretch >= 1";
                    return SLLBM_ERR_ARG;
                }
                std::vector<double> sz;
                for (int k = side; k >= 1; --k) sz.push_back(std::pow(d.stretch, k));
                for (int k = 0; k < nc; ++k) sz.push_back(1.0);
                for (int k = 1; k <= side; ++k) sz.push_back(std::pow(d.stretch, k));
                double tot = 0;
                for (double s : sz) tot += s;
                const double h = L / tot;
                V[0] = -0.5 * L;
                double acc = 0;
                for (int j = 0; j < C; ++j) {
                    acc += sz[j] * h;
                    V[j + 1] = acc - 0.5 * L;
                }
            }
        }
        for (int64_t n = 0; n < m.n_nodes; ++n) {
            int64_t r = n;
            for (int dd = 0; dd < D; ++dd) {
                const int k = int(r % m.N[dd]);
                r /= m.N[dd];
                auto cl = node_logical(dd, k);
                const auto& V = m.V[dd];
                m.X[n * D + dd] = V[cl.first] + cl.second * (V[cl.first + 1] - V[cl.first]);
            }
        }
    } else {
        const int Ca = m.cells[0], Cr = m.cells[1];
        const double R = m.length[1];
        const double q = d.stretch;
        if (!(q > 1.0) || !(R > 1.0) || !(d.thickness > 0 && d.thickness < 0.5)) {
            err = "NACA mesh: stretch > 1, radius > 1, 0 < thickness < 0.5";
            return SLLBM_ERR_ARG;
        }
        for (int64_t n = 0; n < m.n_nodes; ++n) {
            const int ka = int(n % m.N[0]);
            const int kb = int(n / m.N[0]);
            auto la = node_logical(0, ka);
            auto lb = node_logical(1, kb);
            const double s = la.first + la.second;
            const double r = lb.first + lb.second;
            const double ang = 2.0 * kPi * s / Ca;
            // cosine clustering at the leading edge, linear start at the trailing edge
            const double psi = 0.5 * (1.0 - std::cos(ang)) + 0.25 * std::fabs(std::sin(ang)) * 0.5 * (1.0 + std::cos(ang));
            const double xs = 1.0 - psi;
            const double ys = (std::sin(ang) >= 0.0 ? 1.0 : -1.0) * naca_half(xs, d.thickness);
            const double xf = 0.5 + R * std::cos(ang), yf = R * std::sin(ang);
            const double fr = (std::pow(q, r) - 1.0) / (std::pow(q, double(Cr)) - 1.0);
            m.X[n * 2 + 0] = xs + fr * (xf - xs);
            m.X[n * 2 + 1] = ys + fr * (yf - ys);
        }
    }
    return SLLBM_OK;
}

}  // namespace sllbm
