// Recursive bipartite scene splitting (Sec. 3.2 "Scene Splitting", Alg. 1)
// and the overlap by a box scale factor s (Sec. 3.2; s = 1.4 in Sec. 4).
//
// Host pre-processing, run once before training: it turns a point cloud
// (and the training cameras) into the K block-local sets whose shared
// members are the Gaussians the consensus averages.
//
// The split works on ground-plane positions (x, y): the scene has one axis
// aligned to the ground and blocks are ground cells spanning the full
// height.  Each cell carries a budget of leaves; a cell with budget k >= 2
// is split on the longer side of the tight box of its points, the first
// floor(n k_lo / k) points in (coordinate, index) order going to the lower
// child with budget k_lo = floor(k / 2).  Cells are processed level by level
// in first-in first-out order, as Alg. 1 pops and pushes them, so for K a
// power of two this is Alg. 1 with a median cut, and every other K still
// gets blocks of equal size up to one point.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <deque>
#include <limits>
#include <vector>

#include "dogs.h"

namespace {

struct Cell {
    std::vector<int64_t> pts;
    int budget;
};

void tight_box(const double* xy, const std::vector<int64_t>& pts, double* box) {
    const double inf = std::numeric_limits<double>::infinity();
    double b[4] = {inf, -inf, inf, -inf};
    for (int64_t i : pts) {
        const double x = xy[2 * i], y = xy[2 * i + 1];
        b[0] = std::min(b[0], x);
        b[1] = std::max(b[1], x);
        b[2] = std::min(b[2], y);
        b[3] = std::max(b[3], y);
    }
    for (int j = 0; j < 4; ++j) box[j] = b[j];
}

bool finite_xy(const double* xy, int64_t n) {
    for (int64_t i = 0; i < 2 * n; ++i)
        if (!std::isfinite(xy[i])) return false;
    return true;
}

// squared distance from (x, y) to a box; 0 inside
double box_dist2(const double* b, double x, double y) {
    const double dx = x < b[0] ? b[0] - x : (x > b[1] ? x - b[1] : 0.0);
    const double dy = y < b[2] ? b[2] - y : (y > b[3] ? y - b[3] : 0.0);
    return dx * dx + dy * dy;
}

}  // namespace

extern "C" int dg_scene_split(const double* xy, int64_t n, int K, int32_t* cell, double* boxes) {
    if (K < 1 || K > DG_MAX_BLOCKS || n < 0 || !boxes || (n > 0 && (!xy || !cell))) return DG_ERR_INVALID;
    if (!finite_xy(xy, n)) return DG_ERR_INVALID;
    std::deque<Cell> cells;
    {
        Cell root;
        root.pts.resize(n);
        for (int64_t i = 0; i < n; ++i) root.pts[i] = i;
        root.budget = K;
        cells.push_back(std::move(root));
    }
    // one pass over the current cells per level; leaves (budget 1) are
    // re-queued untouched so the final order is the order of Alg. 1
    while ((int)cells.size() < K) {
        const size_t level = cells.size();
        for (size_t c = 0; c < level; ++c) {
            Cell cur = std::move(cells.front());
            cells.pop_front();
            if (cur.budget < 2) {
                cells.push_back(std::move(cur));
                continue;
            }
            double b[4];
            tight_box(xy, cur.pts, b);
            // longer side; an empty cell or a tie cuts along x
            const int axis = (cur.pts.empty() || b[1] - b[0] >= b[3] - b[2]) ? 0 : 1;
            std::sort(cur.pts.begin(), cur.pts.end(), [&](int64_t a, int64_t bb) {
                const double ca = xy[2 * a + axis], cb = xy[2 * bb + axis];
                return ca < cb || (ca == cb && a < bb);
            });
            const int k_lo = cur.budget / 2;
            const int64_t m = (int64_t)cur.pts.size() * k_lo / cur.budget;
            Cell lo, hi;
            lo.pts.assign(cur.pts.begin(), cur.pts.begin() + m);
            hi.pts.assign(cur.pts.begin() + m, cur.pts.end());
            lo.budget = k_lo;
            hi.budget = cur.budget - k_lo;
            cells.push_back(std::move(lo));
            cells.push_back(std::move(hi));
        }
    }
    for (int k = 0; k < K; ++k) {
        tight_box(xy, cells[k].pts, boxes + 4 * k);
        for (int64_t i : cells[k].pts) cell[i] = k;
    }
    return DG_OK;
}

extern "C" int dg_scene_assign(const double* xy, int64_t n, const double* boxes, int K, double s,
                               const int32_t* own, int nearest, uint64_t* member) {
    if (K < 1 || K > DG_MAX_BLOCKS || n < 0 || !boxes || !(s >= 1.0) || !std::isfinite(s) ||
        (n > 0 && (!xy || !member)))
        return DG_ERR_INVALID;
    if (!finite_xy(xy, n)) return DG_ERR_INVALID;
    if (own)
        for (int64_t i = 0; i < n; ++i)
            if (own[i] < 0 || own[i] >= K) return DG_ERR_INVALID;
    // expanded boxes: same centre, sides scaled by s; an empty box stays empty
    std::vector<double> ex(4 * (size_t)K);
    std::vector<char> empty(K);
    for (int k = 0; k < K; ++k) {
        const double* b = boxes + 4 * k;
        empty[k] = !(b[0] <= b[1] && b[2] <= b[3]);
        for (int a = 0; a < 2; ++a) {
            const double lo = b[2 * a], hi = b[2 * a + 1];
            const double c = 0.5 * (lo + hi), h = 0.5 * s * (hi - lo);
            ex[4 * k + 2 * a] = c - h;
            ex[4 * k + 2 * a + 1] = c + h;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        const double x = xy[2 * i], y = xy[2 * i + 1];
        uint64_t m = own ? (uint64_t(1) << own[i]) : 0;
        for (int k = 0; k < K; ++k) {
            const double* e = &ex[4 * k];
            if (!empty[k] && x >= e[0] && x <= e[1] && y >= e[2] && y <= e[3]) m |= uint64_t(1) << k;
        }
        if (m == 0 && nearest) {
            int best = -1;
            double bd = 0.0;
            for (int k = 0; k < K; ++k) {
                if (empty[k]) continue;
                const double d = box_dist2(&ex[4 * k], x, y);
                if (best < 0 || d < bd) best = k, bd = d;
            }
            if (best >= 0) m = uint64_t(1) << best;
        }
        member[i] = m;
    }
    return DG_OK;
}
