// Lattice geometry of quantum Z2 lattice gauge theory (Sec. 2.1): one qubit
// per link of a periodic d-dimensional lattice, N_l = d L^d links and
// N_p = N_l (d - 1) / 2 plaquettes.  Host side; builds the bit masks that the
// kernels and reductions consume.
#include <cstring>

#include "internal.h"

namespace z2 {
namespace {

struct Geo {
    int d;
    int L[3];
    int sites;
    void coords(int s, int c[3]) const {
        for (int mu = 0; mu < 3; ++mu) {
            c[mu] = mu < d ? s % L[mu] : 0;
            if (mu < d) s /= L[mu];
        }
    }
    int site(const int c[3]) const {
        int s = 0;
        for (int mu = d - 1; mu >= 0; --mu) s = s * L[mu] + ((c[mu] % L[mu]) + L[mu]) % L[mu];
        return s;
    }
    int step(int s, int mu, int delta) const {
        int c[3];
        coords(s, c);
        c[mu] += delta;
        return site(c);
    }
    int link(int s, int mu) const { return d * s + mu; }
};

inline uint64_t bit(int l) { return uint64_t(1) << l; }

}  // namespace

bool build_lattice(int d, const int32_t *L, Lattice &out, std::string &err) {
    if (d != 2 && d != 3) {
        err = "lattice dimension must be 2 or 3";
        return false;
    }
    if (!L) {
        err = "lattice sizes are NULL";
        return false;
    }
    Geo g{};
    g.d = d;
    g.sites = 1;
    for (int mu = 0; mu < 3; ++mu) g.L[mu] = 1;
    for (int mu = 0; mu < d; ++mu) {
        if (L[mu] < 2 || L[mu] > 64) {
            err = "every lattice extent must be in [2, 64]";
            return false;
        }
        g.L[mu] = L[mu];
        g.sites *= L[mu];
    }
    const int n_links = d * g.sites;
    if (n_links > Z2_MAX_LINKS) {
        err = "lattice has " + std::to_string(n_links) + " links; at most " +
              std::to_string(Z2_MAX_LINKS) + " qubits are supported";
        return false;
    }
    Lattice lat;
    lat.d = d;
    for (int mu = 0; mu < 3; ++mu) lat.L[mu] = g.L[mu];
    lat.n_sites = g.sites;
    lat.n_links = n_links;

    // plaquettes: site-major, then planes (0,1), (0,2), (1,2)
    for (int s = 0; s < g.sites; ++s)
        for (int mu = 0; mu < d; ++mu)
            for (int nu = mu + 1; nu < d; ++nu) {
                uint64_t m = bit(g.link(s, mu)) | bit(g.link(g.step(s, mu, 1), nu)) |
                             bit(g.link(g.step(s, nu, 1), mu)) | bit(g.link(s, nu));
                lat.plaq.push_back(m);
            }
    lat.n_plaq = (int)lat.plaq.size();
    if (lat.n_plaq > Z2_MAX_PLAQ || g.sites > Z2_MAX_SITES) {
        err = "too many plaquettes or sites";
        return false;
    }
    for (int s = 0; s < g.sites; ++s) {
        uint64_t m = 0;
        for (int mu = 0; mu < d; ++mu) m |= bit(g.link(s, mu)) | bit(g.link(g.step(s, mu, -1), mu));
        lat.star.push_back(m);
    }
    for (int mu = 0; mu < d; ++mu) {
        uint64_t w = 0, v = 0;
        int c[3] = {0, 0, 0};
        for (int k = 0; k < g.L[mu]; ++k) {
            c[mu] = k;
            w |= bit(g.link(g.site(c), mu));
        }
        for (int s = 0; s < g.sites; ++s) {
            int cc[3];
            g.coords(s, cc);
            if (cc[mu] == 0) v |= bit(g.link(s, mu));
        }
        lat.wmu.push_back(w);
        lat.vmu.push_back(v);
    }
    // index of the plaquette (s, mu, nu) in the list above
    auto pidx = [&](int s, int mu, int nu) {
        int per_site = d * (d - 1) / 2;
        int plane = (mu == 0 && nu == 1) ? 0 : (mu == 0 && nu == 2) ? 1 : 2;
        return s * per_site + plane;
    };
    auto at = [&](int x, int y, int z) {
        int c[3] = {x, y, z};
        return g.site(c);
    };
    // 2x2 Wilson loop in the xy plane at the origin = product of 4 plaquettes
    lat.wilson2x2 = lat.plaq[pidx(at(0, 0, 0), 0, 1)] ^ lat.plaq[pidx(at(1, 0, 0), 0, 1)] ^
                    lat.plaq[pidx(at(0, 1, 0), 0, 1)] ^ lat.plaq[pidx(at(1, 1, 0), 0, 1)];
    lat.wilson_degenerate = g.L[0] < 3 || g.L[1] < 3;
    // contours c1, c2, c3 (perimeters 4, 6, 8; Sec. 3.1)
    const uint64_t p00 = lat.plaq[pidx(at(0, 0, 0), 0, 1)];
    if (d == 2) {
        const uint64_t p10 = lat.plaq[pidx(at(1, 0, 0), 0, 1)];
        const uint64_t p01 = lat.plaq[pidx(at(0, 1, 0), 0, 1)];
        lat.contour[0] = p00;
        lat.contour[1] = p00 ^ p10;
        lat.contour[2] = p00 ^ p10 ^ p01;
        lat.contour_degenerate[1] = g.L[0] < 3;
        lat.contour_degenerate[2] = g.L[0] < 3 || g.L[1] < 3;
    } else {
        const uint64_t q = lat.plaq[pidx(at(0, 0, 0), 0, 2)];
        const uint64_t pz = lat.plaq[pidx(at(0, 0, 1), 0, 1)];
        lat.contour[0] = p00;
        lat.contour[1] = p00 ^ q;
        lat.contour[2] = p00 ^ q ^ pz;
    }
    std::memset(lat.colmask, 0, sizeof(lat.colmask));
    for (int p = 0; p < lat.n_plaq; ++p)
        for (int l = 0; l < n_links; ++l)
            if (lat.plaq[p] & bit(l)) lat.colmask[l] |= 1u << p;
    out = std::move(lat);
    return true;
}

}  // namespace z2
