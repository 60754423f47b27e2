// Host-side finite-element assembly (see assembly.h).
#include "assembly.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace daeti {

void conductivity_tensor(double d_long, double d_trans, const double* fibre, int dim, double D[9]) {
    double f[3] = {0, 0, 0};
    double nrm = 0.0;
    if (fibre) {
        for (int d = 0; d < dim; ++d) {
            f[d] = fibre[d];
            nrm += f[d] * f[d];
        }
    }
    nrm = std::sqrt(nrm);
    const double dl = nrm > 0 ? d_long : d_trans;
    if (!fibre) {
        // isotropic d_long when no fibre field is given
        for (int r = 0; r < 9; ++r) D[r] = 0.0;
        for (int d = 0; d < dim; ++d) D[d * 3 + d] = d_long;
        return;
    }
    for (int d = 0; d < dim; ++d) f[d] = nrm > 0 ? f[d] / nrm : 0.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double v = (r == c && r < dim) ? d_trans : 0.0;
            if (r < dim && c < dim) v += (dl - d_trans) * f[r] * f[c];
            D[r * 3 + c] = v;
        }
}

void box_stiffness(int dim, double h, const double D[9], double* Ke) {
    const int nl = 1 << dim;
    const double g[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
    std::memset(Ke, 0, sizeof(double) * nl * nl);
    const int nq = 1 << dim;
    for (int q = 0; q < nq; ++q) {
        double xi[3] = {g[q & 1], g[(q >> 1) & 1], g[(q >> 2) & 1]};
        const double w = std::pow(0.5, dim);
        double grad[8][3];
        for (int a = 0; a < nl; ++a) {
            for (int d = 0; d < dim; ++d) {
                double gd = ((a >> d) & 1) ? 1.0 : -1.0;
                for (int e = 0; e < dim; ++e) {
                    if (e == d) continue;
                    gd *= ((a >> e) & 1) ? xi[e] : 1.0 - xi[e];
                }
                grad[a][d] = gd / h;
            }
        }
        const double jac = std::pow(h, dim);
        for (int a = 0; a < nl; ++a)
            for (int b = 0; b < nl; ++b) {
                double s = 0.0;
                for (int r = 0; r < dim; ++r)
                    for (int c = 0; c < dim; ++c) s += grad[a][r] * D[r * 3 + c] * grad[b][c];
                Ke[a * nl + b] += w * jac * s;
            }
    }
}

double tet_stiffness(const double X[12], const double D[9], double Ke[16]) {
    double J[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) J[r][c] = X[(c + 1) * 3 + r] - X[r];
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    const double vol = std::fabs(det) / 6.0;
    if (!(vol > 0.0)) return 0.0;
    // inverse of J: rows are the gradients of the barycentric coordinates 1..3
    double inv[3][3];
    inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    double G[4][3];
    for (int d = 0; d < 3; ++d) {
        G[1][d] = inv[0][d];
        G[2][d] = inv[1][d];
        G[3][d] = inv[2][d];
        G[0][d] = -(inv[0][d] + inv[1][d] + inv[2][d]);
    }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            double s = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) s += G[a][r] * D[r * 3 + c] * G[b][c];
            Ke[a * 4 + b] = vol * s;
        }
    return vol;
}

static void elem_tensor(int dim, const double* d_long, const double* d_trans, const double* fibre, int64_t e,
                        double D[9]) {
    conductivity_tensor(d_long[e], d_trans[e], fibre ? fibre + 3 * e : nullptr, dim, D);
}

bool grid_layer_stiffness(int dim, const int64_t n[3], double h, const double* d_long, const double* d_trans,
                          const double* fibre, double* layerK) {
    const int64_t nx = n[0], ny = n[1], nz = dim == 3 ? n[2] : 1;
    const int64_t ex_n = nx - 1, ey_n = ny - 1, ez_n = dim == 3 ? nz - 1 : 1;
    const int64_t per_layer = ex_n * ey_n;
    const int nl = 1 << dim;
    const double* dt = d_trans ? d_trans : d_long;
    for (int64_t ez = 0; ez < ez_n; ++ez) {
        const int64_t e0 = ez * per_layer;
        double D0[9];
        elem_tensor(dim, d_long, dt, fibre, e0, D0);
        for (int64_t e = e0 + 1; e < e0 + per_layer; ++e) {
            double D[9];
            elem_tensor(dim, d_long, dt, fibre, e, D);
            for (int r = 0; r < 9; ++r)
                if (D[r] != D0[r]) return false;
        }
        box_stiffness(dim, h, D0, layerK + ez * nl * nl);
    }
    return true;
}

void grid_class_table(int dim, const int64_t n[3], double h, const double* layerK, double* K, double* m) {
    const int64_t nz = dim == 3 ? n[2] : 1;
    const int64_t ez_n = dim == 3 ? nz - 1 : 1;
    const int nl = 1 << dim;
    std::fill(K, K + nz * 9 * 27, 0.0);
    std::fill(m, m + nz * 9, 0.0);
    const double emass = std::pow(h, dim) / nl;
    for (int64_t z = 0; z < nz; ++z)
        for (int cy = 0; cy < 3; ++cy)
            for (int cx = 0; cx < 3; ++cx) {
                const int64_t cls = (z * 3 + cy) * 3 + cx;
                double* Kr = K + cls * 27;
                // adjacent elements: origin offsets ox, oy, oz in {-1, 0}
                for (int oz = (dim == 3 ? -1 : 0); oz <= 0; ++oz) {
                    const int64_t ez = z + oz;
                    if (dim == 3 && (ez < 0 || ez >= ez_n)) continue;
                    const double* Ke = layerK + (dim == 3 ? ez : 0) * nl * nl;
                    for (int oy = -1; oy <= 0; ++oy) {
                        if (oy == -1 && cy == 0) continue;
                        if (oy == 0 && cy == 2) continue;
                        for (int ox = -1; ox <= 0; ++ox) {
                            if (ox == -1 && cx == 0) continue;
                            if (ox == 0 && cx == 2) continue;
                            const int a = (-ox) | ((-oy) << 1) | ((dim == 3 ? -oz : 0) << 2);
                            for (int b = 0; b < nl; ++b) {
                                const int dx = ox + (b & 1), dy = oy + ((b >> 1) & 1);
                                const int dz = dim == 3 ? oz + ((b >> 2) & 1) : 0;
                                Kr[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] += Ke[a * nl + b];
                            }
                            m[cls] += emass;
                        }
                    }
                }
            }
}

bool build_grid_table(int dim, const int64_t n[3], double h, const double* d_long, const double* d_trans,
                      const double* fibre, GridTable& out) {
    const int64_t nz = dim == 3 ? n[2] : 1;
    const int64_t ez_n = dim == 3 ? nz - 1 : 1;
    const int nl = 1 << dim;
    std::vector<double> layerK((size_t)ez_n * nl * nl);
    if (!grid_layer_stiffness(dim, n, h, d_long, d_trans, fibre, layerK.data())) return false;
    out.dim = dim;
    out.nx = (int)n[0];
    out.ny = (int)n[1];
    out.nz = (int)nz;
    out.K.assign((size_t)nz * 9 * 27, 0.0);
    out.m.assign((size_t)nz * 9, 0.0);
    grid_class_table(dim, n, h, layerK.data(), out.K.data(), out.m.data());
    return true;
}

// CSR from element connectivity and per-element matrices produced on the fly.
template <class ElemFn>
static void assemble_csr_generic(int64_t n_nodes, int64_t n_elem, int nl, const int64_t* conn, ElemFn elem,
                                 CsrK& out) {
    // node -> elements
    std::vector<int64_t> cnt(n_nodes + 1, 0);
    for (int64_t e = 0; e < n_elem; ++e)
        for (int a = 0; a < nl; ++a) cnt[conn[e * nl + a] + 1]++;
    for (int64_t i = 0; i < n_nodes; ++i) cnt[i + 1] += cnt[i];
    std::vector<int64_t> ne(cnt[n_nodes]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t e = 0; e < n_elem; ++e)
        for (int a = 0; a < nl; ++a) ne[fill[conn[e * nl + a]]++] = e;
    // pattern
    out.n = n_nodes;
    out.rowptr.assign(n_nodes + 1, 0);
    std::vector<int> buf;
    out.col.clear();
    out.col.reserve((size_t)n_nodes * 16);
    for (int64_t i = 0; i < n_nodes; ++i) {
        buf.clear();
        for (int64_t p = cnt[i]; p < cnt[i + 1]; ++p) {
            const int64_t e = ne[p];
            for (int a = 0; a < nl; ++a) buf.push_back((int)conn[e * nl + a]);
        }
        if (buf.empty()) buf.push_back((int)i);
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        out.col.insert(out.col.end(), buf.begin(), buf.end());
        out.rowptr[i + 1] = (int64_t)out.col.size();
    }
    out.val.assign(out.col.size(), 0.0);
    out.m.assign(n_nodes, 0.0);
    std::vector<double> Ke(nl * nl);
    for (int64_t e = 0; e < n_elem; ++e) {
        const double mass = elem(e, Ke.data());
        for (int a = 0; a < nl; ++a) {
            const int64_t r = conn[e * nl + a];
            out.m[r] += mass / nl;
            const int* cb = out.col.data() + out.rowptr[r];
            const int len = (int)(out.rowptr[r + 1] - out.rowptr[r]);
            for (int b = 0; b < nl; ++b) {
                const int c = (int)conn[e * nl + b];
                const int pos = (int)(std::lower_bound(cb, cb + len, c) - cb);
                out.val[out.rowptr[r] + pos] += Ke[a * nl + b];
            }
        }
    }
}

bool assemble_grid_csr(int dim, const int64_t n[3], double h, const double* d_long, const double* d_trans,
                       const double* fibre, CsrK& out, std::string& err) {
    const int64_t nx = n[0], ny = n[1], nz = dim == 3 ? n[2] : 1;
    const int64_t ex_n = nx - 1, ey_n = ny - 1, ez_n = dim == 3 ? nz - 1 : 1;
    const int nl = 1 << dim;
    const int64_t n_elem = ex_n * ey_n * ez_n;
    std::vector<int64_t> conn((size_t)n_elem * nl);
    for (int64_t ez = 0; ez < ez_n; ++ez)
        for (int64_t ey = 0; ey < ey_n; ++ey)
            for (int64_t ex = 0; ex < ex_n; ++ex) {
                const int64_t e = ex + ex_n * (ey + ey_n * ez);
                for (int a = 0; a < nl; ++a) {
                    const int64_t x = ex + (a & 1), y = ey + ((a >> 1) & 1), z = ez + ((a >> 2) & 1);
                    conn[e * nl + a] = x + nx * (y + ny * (dim == 3 ? z : 0));
                }
            }
    const double vol = std::pow(h, dim);
    assemble_csr_generic(nx * ny * nz, n_elem, nl, conn.data(),
                         [&](int64_t e, double* Ke) {
                             double D[9];
                             elem_tensor(dim, d_long, d_trans, fibre, e, D);
                             box_stiffness(dim, h, D, Ke);
                             return vol;
                         },
                         out);
    (void)err;
    return true;
}

bool assemble_tet_csr(int64_t n_nodes, const double* xyz, int64_t n_tets, const int64_t* tets,
                      const double* d_long, const double* d_trans, const double* fibre, CsrK& out,
                      std::string& err) {
    for (int64_t e = 0; e < n_tets * 4; ++e)
        if (tets[e] < 0 || tets[e] >= n_nodes) {
            err = "tet node index out of range";
            return false;
        }
    bool bad = false;
    assemble_csr_generic(n_nodes, n_tets, 4, tets,
                         [&](int64_t e, double* Ke) {
                             double X[12], D[9];
                             for (int a = 0; a < 4; ++a)
                                 for (int d = 0; d < 3; ++d) X[a * 3 + d] = xyz[tets[e * 4 + a] * 3 + d];
                             elem_tensor(3, d_long, d_trans, fibre, e, D);
                             const double v = tet_stiffness(X, D, Ke);
                             if (!(v > 0.0)) bad = true;
                             return v;
                         },
                         out);
    if (bad) {
        err = "degenerate tetrahedron";
        return false;
    }
    return true;
}

void csr_to_sell32(const CsrK& K, const double* scale, Sell32& out) {
    const int64_t n = K.n;
    out.n_chunks = (n + 31) / 32;
    out.chunk_ptr.assign(out.n_chunks + 1, 0);
    out.chunk_w.assign(out.n_chunks, 0);
    out.diag.assign(n, 0.0);
    for (int64_t c = 0; c < out.n_chunks; ++c) {
        int w = 0;
        for (int64_t r = c * 32; r < std::min<int64_t>(n, c * 32 + 32); ++r) {
            const int len = (int)(K.rowptr[r + 1] - K.rowptr[r]) - 1;   // minus the diagonal
            w = std::max(w, len);
        }
        out.chunk_w[c] = w;
        out.chunk_ptr[c + 1] = out.chunk_ptr[c] + 32 * (int64_t)w;
    }
    out.col.assign(out.chunk_ptr[out.n_chunks], 0);
    out.val.assign(out.chunk_ptr[out.n_chunks], 0.0);
    for (int64_t c = 0; c < out.n_chunks; ++c) {
        for (int lane = 0; lane < 32; ++lane) {
            const int64_t r = c * 32 + lane;
            const int64_t base = out.chunk_ptr[c] + lane;
            int j = 0;
            if (r < n) {
                const double s = scale ? scale[r] : 1.0;
                for (int64_t p = K.rowptr[r]; p < K.rowptr[r + 1]; ++p) {
                    if (K.col[p] == r) {
                        out.diag[r] = K.val[p];
                        continue;
                    }
                    out.col[base + 32 * (int64_t)j] = K.col[p];
                    out.val[base + 32 * (int64_t)j] = K.val[p] * s;
                    ++j;
                }
            }
            for (; j < out.chunk_w[c]; ++j) {
                out.col[base + 32 * (int64_t)j] = (int)std::min<int64_t>(r, n - 1);
                out.val[base + 32 * (int64_t)j] = 0.0;
            }
        }
    }
}

}  // namespace daeti
