// btdf_tables.cu - host-side construction of the static immersed-boundary
// tables of one lattice: per-marker support and weights (Eq. 14, FP64
// evaluation of the delta functions of Eqs. 37-39), and the node-centric
// spreading table (Eq. 15) over 128-node band segments.  Shared by the
// single-lattice context and the batched form.
#include "btdf_internal.cuh"

#include <algorithm>
#include <cmath>

namespace btdf {

double delta_fn(int kind, double r) {
    const double a = std::fabs(r);
    switch (kind) {
    case 2:  // Eq. 37
        return a <= 1.0 ? 1.0 - a : 0.0;
    case 3:  // Eq. 38
        if (a > 1.5) return 0.0;
        if (a > 0.5) return (5.0 - 3.0 * a - std::sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a))) / 6.0;
        return (1.0 + std::sqrt(1.0 - 3.0 * a * a)) / 3.0;
    case 4:  // Eq. 39
        if (a >= 2.0) return 0.0;
        if (a >= 1.0) return (5.0 - 2.0 * a - std::sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
        return (3.0 - 2.0 * a + std::sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    case 5:  // cosine kernel with 4-point support
        return a < 2.0 ? 0.25 * (1.0 + std::cos(M_PI * a * 0.5)) : 0.0;
    default:
        return 0.0;
    }
}

// d delta / dr of the same functions (Eqs. 37-39 differentiated; the 2-point
// kernel takes the one-sided slope at its kinks).
double delta_deriv(int kind, double r) {
    const double a = std::fabs(r), sg = r < 0.0 ? -1.0 : 1.0;
    switch (kind) {
    case 2:
        return a < 1.0 ? -sg : 0.0;
    case 3:
        if (a >= 1.5) return 0.0;
        if (a > 0.5) return sg * (-0.5 - (1.0 - a) / (2.0 * std::sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a))));
        return sg * (-a / std::sqrt(1.0 - 3.0 * a * a));
    case 4:
        if (a >= 2.0) return 0.0;
        if (a >= 1.0) return sg * (-2.0 - (6.0 - 4.0 * a) / std::sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
        return sg * (-2.0 + (2.0 - 4.0 * a) / std::sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    case 5:
        return a < 2.0 ? -sg * (M_PI / 8.0) * std::sin(M_PI * a * 0.5) : 0.0;
    default:
        return 0.0;
    }
}

void build_adjoint_markers(int nx, int ny, int delta, int width, bool px, bool py,
                           const std::vector<BodyDesc>& bodies, std::vector<AdjMarker>& out) {
    const int S = width;
    out.clear();
    for (const BodyDesc& B : bodies)
        for (int l = 0; l < B.n; l++) {
            const double X = B.X[l], Y = B.Y[l];
            const int i0 = (int)std::floor(X - 0.5 * S) + 1;
            const int j0 = (int)std::floor(Y - 0.5 * S) + 1;
            AdjMarker A{};
            for (int i = 0; i < S; i++) {
                int x = i0 + i, y = j0 + i;
                if (px) x = ((x % nx) + nx) % nx;
                if (py) y = ((y % ny) + ny) % ny;
                if (x >= 0 && x < nx) {
                    A.wx[i] = (float)delta_fn(delta, (double)(i0 + i) - X);
                    A.dwx[i] = (float)(-delta_deriv(delta, (double)(i0 + i) - X));   // d/dX
                }
                if (y >= 0 && y < ny) {
                    A.wy[i] = (float)delta_fn(delta, (double)(j0 + i) - Y);
                    A.dwy[i] = (float)(-delta_deriv(delta, (double)(j0 + i) - Y));
                }
            }
            out.push_back(A);
        }
}

void build_marker_tables(int nx, int ny, int nseg, int delta, int width, bool px, bool py,
                         double u_in, const std::vector<BodyDesc>& bodies, int marker_base,
                         HostTables& t) {
    const int S = width;
    int nm = 0;
    for (const BodyDesc& B : bodies) nm += B.n;
    t.mk.assign(nm, Marker{});
    t.aux.assign(nm, MarkerAux{});
    t.wsum.assign(nm, 0.0);
    struct Ent {
        long long node;
        int marker;
        double w;
    };
    std::vector<Ent> ents;
    ents.reserve((size_t)nm * S * S);
    int m = 0;
    for (const BodyDesc& B : bodies) {
        for (int l = 0; l < B.n; l++, m++) {
            const double X = B.X[l], Y = B.Y[l];
            const int i0 = (int)std::floor(X - 0.5 * S) + 1;   // first node with x > X - S/2
            const int j0 = (int)std::floor(Y - 0.5 * S) + 1;
            double wx[4] = {0, 0, 0, 0}, wy[4] = {0, 0, 0, 0};
            bool okx[4] = {false, false, false, false}, oky[4] = {false, false, false, false};
            Marker& M = t.mk[m];
            for (int i = 0; i < 4; i++) {
                M.xs[i] = 0;
                M.ys[i] = 0;
            }
            for (int i = 0; i < S; i++) {
                int x = i0 + i, y = j0 + i;
                wx[i] = delta_fn(delta, (double)x - X);
                wy[i] = delta_fn(delta, (double)y - Y);
                if (px) x = ((x % nx) + nx) % nx;
                if (py) y = ((y % ny) + ny) % ny;
                okx[i] = x >= 0 && x < nx;
                oky[i] = y >= 0 && y < ny;
                M.xs[i] = std::min(std::max(x, 0), nx - 1);
                M.ys[i] = std::min(std::max(y, 0), ny - 1);
            }
            for (int k = 0; k < 16; k++) M.w[k] = 0.0f;
            for (int j = 0; j < S; j++)
                for (int i = 0; i < S; i++) {
                    if (!okx[i] || !oky[j]) continue;
                    const double w = wx[i] * wy[j];
                    M.w[j * S + i] = (float)w;
                    t.wsum[m] += w;
                    if (w != 0.0)
                        ents.push_back({(long long)M.ys[j] * nx + M.xs[i], marker_base + m,
                                        w * B.drs * B.ds});
                }
            MarkerAux& A = t.aux[m];
            A.wsum = (float)t.wsum[m];
            A.ubx_rel = (float)((B.Ubx ? B.Ubx[l] : 0.0) - u_in * t.wsum[m]);
            A.uby_rel = (float)(B.Uby ? B.Uby[l] : 0.0);
            A.body = B.tag;
        }
    }
    std::sort(ents.begin(), ents.end(), [](const Ent& a, const Ent& b) {
        return a.node != b.node ? a.node < b.node : a.marker < b.marker;
    });
    // Band segments: 128-node runs of a row holding at least one band node.
    t.seg_index.assign((size_t)ny * nseg, -1);
    t.seg_keys.clear();
    for (const Ent& e : ents) {
        const long long y = e.node / nx, x = e.node % nx;
        const long long key = y * nseg + x / kSeg;
        if (t.seg_keys.empty() || t.seg_keys.back() != key) t.seg_keys.push_back(key);
    }
    const int nband = (int)t.seg_keys.size();
    for (int s = 0; s < nband; s++) t.seg_index[t.seg_keys[s]] = s;
    t.seg_ptr.assign((size_t)nband * (kSeg + 1), 0);
    t.csr.assign(ents.size(), CsrEntry{});
    // entries are sorted by node, so each segment's entries are contiguous
    size_t k = 0;
    for (int s = 0; s < nband; s++) {
        const long long key = t.seg_keys[s];
        const long long y = key / nseg, xs0 = (key % nseg) * kSeg;
        int* ptr = &t.seg_ptr[(size_t)s * (kSeg + 1)];
        for (int i = 0; i < kSeg; i++) {
            ptr[i] = (int)k;
            const long long node = y * nx + xs0 + i;
            while (k < ents.size() && ents[k].node == node && xs0 + i < nx) {
                t.csr[k].marker = ents[k].marker;
                t.csr[k].w = (float)ents[k].w;
                k++;
            }
        }
        ptr[kSeg] = (int)k;
    }
}

}  // namespace btdf
