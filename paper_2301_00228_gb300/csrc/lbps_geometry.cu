// Boundary cells of a rectangle with a circular hole (lbps_disk_cells in
// include/lbps.h): host code only.
//
// The paper builds the cell of a boundary point as the square of side dh
// around it "modified to match the boundary geometry" (Sec. 3,
// preprocessing; Sec. 3.1.1, Eq. contBalanceOfMomentum and Eq. acc_neumann
// need its volume V_C, the lengths l_kr of its faces towards neighbours and
// the external boundary dC_ext).  For the plate with a hole of Sec. 4 this
// library takes the square, clipped to the body rectangle, minus the disk.
//
// Areas: area(S minus D) = area(S) - area(S and D), the second integrated
// over x column by column: at abscissa x (relative to the centre) the disk
// spans (-h(x), h(x)), h = sqrt(r^2 - x^2), so its part inside the
// rectangle's rows [Y0, Y1] is min(Y1, h) - max(Y0, -h) when positive.
// Between the abscissae where h crosses Y0 or Y1 or vanishes, each bound is
// either a constant or +-h, and the integral of h over such a piece is the
// trapezoid under its chord plus the circular segment between chord and arc.
// Side lengths: the side's length minus its overlap with the chord of the
// disk on its line.
#include <algorithm>
#include <cmath>
#include <initializer_list>

#include "lbps.h"

namespace {

double chord_height(double x, double r) { return std::sqrt(std::max((r - x) * (r + x), 0.0)); }

// Integral of h(x) = sqrt(r^2 - x^2) over [a, b] (a < b, both in [-r, r]):
// the trapezoid under the chord from (a, h(a)) to (b, h(b)) plus the
// circular segment above it, r^2 (t - sin t) / 2 with t the angle the chord
// subtends at the centre (the upper half circle is concave).
double h_integral(double a, double b, double r) {
    const double ha = chord_height(a, r), hb = chord_height(b, r);
    const double dx = b - a;
    // h(b) - h(a) = (a - b)(a + b) / (h(a) + h(b)), free of cancellation
    const double dh = ha + hb > 0.0 ? (a - b) * (a + b) / (ha + hb) : 0.0;
    const double chord = std::sqrt(dx * dx + dh * dh);
    const double t = 2.0 * std::asin(std::min(1.0, chord / (2.0 * r)));
    // t - sin t; its Taylor series where the difference would cancel
    const double t2 = t * t;
    const double tms = t < 1e-2 ? t * t2 / 6.0 * (1.0 - t2 / 20.0 * (1.0 - t2 / 42.0)) : t - std::sin(t);
    return 0.5 * (ha + hb) * dx + 0.5 * r * r * tms;
}

// Area of the rectangle [x0, x1] x [y0, y1] inside the open disk of centre
// (cx, cy), radius r.
double rect_in_disk(double x0, double x1, double y0, double y1, double cx, double cy, double r) {
    if (!(r > 0.0) || !(x1 > x0) || !(y1 > y0)) return 0.0;
    x0 -= cx;
    x1 -= cx;
    const double Y0 = y0 - cy, Y1 = y1 - cy;
    // abscissae where the bounds change: the disk's ends, and where h = |Y0|, |Y1|
    double cut[8];
    int n = 0;
    cut[n++] = x0;
    cut[n++] = x1;
    cut[n++] = -r;
    cut[n++] = r;
    for (double Y : {Y0, Y1})
        if (std::fabs(Y) < r) {
            const double w = chord_height(Y, r);
            cut[n++] = -w;
            cut[n++] = w;
        }
    std::sort(cut, cut + n);
    double area = 0.0;
    for (int q = 0; q + 1 < n; ++q) {
        const double a = std::max(cut[q], x0), b = std::min(cut[q + 1], x1);
        if (!(b > a)) continue;
        const double m = 0.5 * (a + b);
        if (std::fabs(m) >= r) continue;
        const double hm = chord_height(m, r);
        if (std::min(Y1, hm) <= std::max(Y0, -hm)) continue;  // the column misses the rows
        const bool top_arc = hm < Y1, bottom_arc = -hm > Y0;
        const double hi = top_arc || bottom_arc ? h_integral(std::max(a, -r), std::min(b, r), r) : 0.0;
        const double top = top_arc ? hi : Y1 * (b - a);
        const double bottom = bottom_arc ? -hi : Y0 * (b - a);
        area += top - bottom;
    }
    return std::min(std::max(area, 0.0), (x1 - x0) * (y1 - y0));
}

// Length of the segment {x = c} x [lo, hi] (or {y = c} x [lo, hi]) outside
// the open disk: d is the distance of the segment's line from the centre,
// m the centre's coordinate along the segment.
double outside_length(double lo, double hi, double d, double m, double r) {
    const double len = hi - lo;
    if (!(len > 0.0)) return 0.0;
    if (!(r > 0.0) || std::fabs(d) >= r) return len;
    const double w = std::sqrt(r * r - d * d);
    const double in = std::max(0.0, std::min(hi, m + w) - std::max(lo, m - w));
    return len - in;
}

}  // namespace

extern "C" int lbps_disk_cells(int32_t nx, int32_t ny, double dh, double cx, double cy, double r,
                               const int32_t edge_type[4], const double edge_value[8], uint8_t* node_type,
                               double* bc_value, double* cell) {
    if (nx < 3 || ny < 3 || !(dh > 0.0) || !std::isfinite(dh) || !std::isfinite(cx) || !std::isfinite(cy) ||
        !std::isfinite(r) || r < 0.0 || !edge_type || !edge_value || !node_type || !bc_value || !cell)
        return LBPS_ERR_INVALID;
    for (int e = 0; e < 4; ++e) {
        if (edge_type[e] != LBPS_NEUMANN && edge_type[e] != LBPS_DIRICHLET) return LBPS_ERR_INVALID;
        if (!std::isfinite(edge_value[2 * e]) || !std::isfinite(edge_value[2 * e + 1])) return LBPS_ERR_INVALID;
    }
    const size_t n = (size_t)nx * (size_t)ny;
    const double Lx = (nx - 1) * dh, Ly = (ny - 1) * dh, half = 0.5 * dh;
    auto in_disk = [&](int i, int j) {
        const double x = i * dh - cx, y = j * dh - cy;
        return x * x + y * y < r * r;
    };
    auto body = [&](int i, int j) { return i >= 0 && i < nx && j >= 0 && j < ny && !in_disk(i, j); };
    std::fill(bc_value, bc_value + 2 * n, 0.0);
    std::fill(cell, cell + 5 * n, 0.0);
    const int DI[4] = {1, 0, -1, 0}, DJ[4] = {0, 1, 0, -1};
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            const size_t k = (size_t)j * nx + i;
            if (!body(i, j)) {
                node_type[k] = LBPS_VOID;
                continue;
            }
            bool boundary = false;
            for (int d = 0; d < 4; ++d) boundary = boundary || !body(i + DI[d], j + DJ[d]);
            if (!boundary) {
                node_type[k] = LBPS_INTERIOR;
                continue;
            }
            // outer edges through the point: bottom, right, top, left
            const bool on[4] = {j == 0, i == nx - 1, j == ny - 1, i == 0};
            int n_dir = 0;
            for (int e = 0; e < 4; ++e) n_dir += on[e] && edge_type[e] == LBPS_DIRICHLET;
            if (n_dir > 0) {  // Dirichlet dominates; mean u* where two meet
                node_type[k] = LBPS_DIRICHLET;
                for (int e = 0; e < 4; ++e)
                    if (on[e] && edge_type[e] == LBPS_DIRICHLET) {
                        bc_value[2 * k] += edge_value[2 * e] / n_dir;
                        bc_value[2 * k + 1] += edge_value[2 * e + 1] / n_dir;
                    }
                continue;
            }
            node_type[k] = LBPS_NEUMANN;
            const double x = i * dh, y = j * dh;
            const double x0 = std::max(x - half, 0.0), x1 = std::min(x + half, Lx);
            const double y0 = std::max(y - half, 0.0), y1 = std::min(y + half, Ly);
            double* c = cell + 5 * k;
            c[0] = (x1 - x0) * (y1 - y0) - rect_in_disk(x0, x1, y0, y1, cx, cy, r);
            // the clipped square's sides E, N, W, S outside the disk
            const double side[4] = {outside_length(y0, y1, x1 - cx, cy, r), outside_length(x0, x1, y1 - cy, cx, r),
                                    outside_length(y0, y1, x0 - cx, cy, r), outside_length(x0, x1, y0 - cy, cx, r)};
            // a side inside the body rectangle faces a neighbour's cell; one
            // on an outer edge is an external face carrying that edge's traction
            const bool inner[4] = {x + half <= Lx, y + half <= Ly, x - half >= 0.0, y - half >= 0.0};
            const int edge_of_side[4] = {1, 2, 3, 0};
            for (int q = 0; q < 4; ++q) {
                if (inner[q]) {
                    c[1 + q] = side[q];
                } else {
                    const int e = edge_of_side[q];
                    bc_value[2 * k] += edge_value[2 * e] * side[q];
                    bc_value[2 * k + 1] += edge_value[2 * e + 1] * side[q];
                }
            }
        }
    }
    return LBPS_OK;
}
