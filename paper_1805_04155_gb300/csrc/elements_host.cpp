// Reference-element tables for the geometry kernel: gradients of the basis
// functions at the quadrature points and the quadrature weights.
//
// 3D elements and rules follow the Appendix: P1 tetrahedron (1 point,
// w = 1/6), P2 tetrahedron (10 nodes, midpoints ordered 12, 23, 13, 24, 34, 14;
// 11-point degree-4 rule with w = -74/5625, 343/45000, 56/2250), Q1
// hexahedron (2x2x2 Gauss), 20-node Q2 hexahedron (3x3x3 Gauss).  2D: P1
// triangle (1 point), P2 triangle (midpoints 12, 23, 13; 7-point degree-5
// rule), Q1 quadrilateral (2x2 Gauss), 8-node serendipity Q2 (3x3 Gauss).
// Point order: simplices as listed; tensor rules with xi_1 fastest.
#include <cmath>
#include <vector>

#include "ep_internal.h"

namespace ep {
namespace {

struct Rule {
    std::vector<double> pts;  // [n_q][dim]
    std::vector<double> w;
};

void gauss1d(int n, std::vector<double>& x, std::vector<double>& w) {
    if (n == 2) {
        const double g = 1.0 / std::sqrt(3.0);
        x = {-g, g};
        w = {1.0, 1.0};
    } else {
        const double g = std::sqrt(0.6);
        x = {-g, 0.0, g};
        w = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    }
}

Rule tensor_rule(int n, int dim) {
    std::vector<double> x, w;
    gauss1d(n, x, w);
    Rule r;
    if (dim == 2) {
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                r.pts.insert(r.pts.end(), {x[i], x[j]});
                r.w.push_back(w[i] * w[j]);
            }
    } else {
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    r.pts.insert(r.pts.end(), {x[i], x[j], x[k]});
                    r.w.push_back(w[i] * w[j] * w[k]);
                }
    }
    return r;
}

Rule simplex_rule(int family, int dim) {
    Rule r;
    if (dim == 2) {
        if (family == EP_P1) {
            r.pts = {1.0 / 3.0, 1.0 / 3.0};
            r.w = {0.5};
        } else {
            const double s = std::sqrt(15.0);
            const double a1 = (6.0 - s) / 21.0, b1 = (9.0 + 2.0 * s) / 21.0;
            const double a2 = (6.0 + s) / 21.0, b2 = (9.0 - 2.0 * s) / 21.0;
            const double w1 = (155.0 - s) / 2400.0, w2 = (155.0 + s) / 2400.0;
            r.pts = {1.0 / 3.0, 1.0 / 3.0, a1, a1, b1, a1, a1, b1, a2, a2, b2, a2, a2, b2};
            r.w = {9.0 / 80.0, w1, w1, w1, w2, w2, w2};
        }
    } else {
        if (family == EP_P1) {
            r.pts = {0.25, 0.25, 0.25};
            r.w = {1.0 / 6.0};
        } else {
            const double a = 1.0 / 14.0, b = 11.0 / 14.0;
            const double t = std::sqrt(5.0 / 14.0);
            const double c = (1.0 + t) / 4.0, d = (1.0 - t) / 4.0;
            r.pts = {0.25, 0.25, 0.25, a, a, a, b, a, a, a, b, a, a, a, b,
                     c, d, d, d, c, d, d, d, c, c, c, d, c, d, c, d, c, c};
            r.w = {-74.0 / 5625.0};
            for (int i = 0; i < 4; ++i) r.w.push_back(343.0 / 45000.0);
            for (int i = 0; i < 6; ++i) r.w.push_back(56.0 / 2250.0);
        }
    }
    return r;
}

// Gradient of all basis functions at one point: out[p*dim + i] = d(phi_p)/d(xi_i).
void grad(int family, int dim, const double* xi, std::vector<double>& out) {
    out.clear();
    if (dim == 2) {
        const double x = xi[0], y = xi[1];
        if (family == EP_P1) {
            out = {-1, -1, 1, 0, 0, 1};
        } else if (family == EP_P2) {
            const double l0 = 1 - x - y;
            // vertices: l(2l-1); edges 4 l_a l_b, derivatives of l0 = (-1,-1), l1 = (1,0), l2 = (0,1)
            const double d0 = 4 * l0 - 1;
            out = {-d0, -d0,
                   4 * x - 1, 0,
                   0, 4 * y - 1,
                   4 * (l0 - x), -4 * x,
                   4 * y, 4 * x,
                   -4 * y, 4 * (l0 - y)};
        } else if (family == EP_Q1) {
            const int sx[4] = {-1, 1, 1, -1}, sy[4] = {-1, -1, 1, 1};
            for (int p = 0; p < 4; ++p) {
                out.push_back(0.25 * sx[p] * (1 + sy[p] * y));
                out.push_back(0.25 * sy[p] * (1 + sx[p] * x));
            }
        } else {
            const int sx[8] = {-1, 1, 1, -1, 0, 1, 0, -1}, sy[8] = {-1, -1, 1, 1, -1, 0, 1, 0};
            for (int p = 0; p < 8; ++p) {
                const double a = sx[p], b = sy[p];
                if (p < 4) {
                    // phi = (1+ax)(1+by)(ax+by-1)/4
                    const double fx = 1 + a * x, fy = 1 + b * y, s = a * x + b * y - 1;
                    out.push_back(0.25 * a * fy * (s + fx));
                    out.push_back(0.25 * b * fx * (s + fy));
                } else if (a == 0) {
                    // phi = (1-x^2)(1+by)/2
                    out.push_back(-x * (1 + b * y));
                    out.push_back(0.5 * b * (1 - x * x));
                } else {
                    out.push_back(0.5 * a * (1 - y * y));
                    out.push_back(-y * (1 + a * x));
                }
            }
        }
        return;
    }
    const double x = xi[0], y = xi[1], z = xi[2];
    if (family == EP_P1) {
        out = {-1, -1, -1, 1, 0, 0, 0, 1, 0, 0, 0, 1};
    } else if (family == EP_P2) {
        const double l[4] = {1 - x - y - z, x, y, z};
        // dl[k][i] = d l_k / d xi_i
        const double dl[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int k = 0; k < 4; ++k)
            for (int i = 0; i < 3; ++i) out.push_back((4 * l[k] - 1) * dl[k][i]);
        const int ea[6] = {0, 1, 0, 1, 2, 0}, eb[6] = {1, 2, 2, 3, 3, 3};
        for (int e = 0; e < 6; ++e)
            for (int i = 0; i < 3; ++i) out.push_back(4 * (dl[ea[e]][i] * l[eb[e]] + l[ea[e]] * dl[eb[e]][i]));
    } else {
        const int cx[20] = {-1, 1, 1, -1, -1, 1, 1, -1, 0, 1, 0, -1, 0, 1, 0, -1, -1, 1, 1, -1};
        const int cy[20] = {-1, -1, 1, 1, -1, -1, 1, 1, -1, 0, 1, 0, -1, 0, 1, 0, -1, -1, 1, 1};
        const int cz[20] = {-1, -1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 1, 1, 1, 1, 0, 0, 0, 0};
        const int np = family == EP_Q1 ? 8 : 20;
        for (int p = 0; p < np; ++p) {
            const double a = cx[p], b = cy[p], c = cz[p];
            if (family == EP_Q1) {
                out.push_back(0.125 * a * (1 + b * y) * (1 + c * z));
                out.push_back(0.125 * b * (1 + a * x) * (1 + c * z));
                out.push_back(0.125 * c * (1 + a * x) * (1 + b * y));
            } else if (p < 8) {
                // phi = (1+ax)(1+by)(1+cz)(ax+by+cz-2)/8
                const double fx = 1 + a * x, fy = 1 + b * y, fz = 1 + c * z, s = a * x + b * y + c * z - 2;
                out.push_back(0.125 * a * fy * fz * (s + fx));
                out.push_back(0.125 * b * fx * fz * (s + fy));
                out.push_back(0.125 * c * fx * fy * (s + fz));
            } else if (a == 0) {
                // phi = (1-x^2)(1+by)(1+cz)/4
                out.push_back(-0.5 * x * (1 + b * y) * (1 + c * z));
                out.push_back(0.25 * b * (1 - x * x) * (1 + c * z));
                out.push_back(0.25 * c * (1 - x * x) * (1 + b * y));
            } else if (b == 0) {
                out.push_back(0.25 * a * (1 - y * y) * (1 + c * z));
                out.push_back(-0.5 * y * (1 + a * x) * (1 + c * z));
                out.push_back(0.25 * c * (1 + a * x) * (1 - y * y));
            } else {
                out.push_back(0.25 * a * (1 + b * y) * (1 - z * z));
                out.push_back(0.25 * b * (1 + a * x) * (1 - z * z));
                out.push_back(-0.5 * z * (1 + a * x) * (1 + b * y));
            }
        }
    }
}

}  // namespace

void reference_tables(int family, int dim, std::vector<double>& dhat, std::vector<double>& wq) {
    Rule r;
    if (family == EP_P1 || family == EP_P2) r = simplex_rule(family, dim);
    else r = tensor_rule(family == EP_Q1 ? 2 : 3, dim);
    wq = r.w;
    dhat.clear();
    std::vector<double> g;
    for (size_t q = 0; q < r.w.size(); ++q) {
        grad(family, dim, &r.pts[q * dim], g);
        dhat.insert(dhat.end(), g.begin(), g.end());
    }
}

}  // namespace ep
