"""Periodic hypercubic lattices for Z2 lattice gauge theory (oracle side).

TEST INFRASTRUCTURE ONLY: used by the test-suite, the smoke check and the
CPU-baseline leg of the benchmark.  Written independently of the product's
own lattice builder (the two share no code); the tests compare them bit for
bit.

Convention (the paper's Fig. 1 numbering is only partly recoverable, so the
library fixes its own and exports a map to the paper's 2D numbering):

* site  s = x + Lx*(y + Ly*z)
* link  l(s, mu) = d*s + mu, mu = 0 (+x), 1 (+y), 2 (+z); qubit l is bit l
* plaquette (s, mu<nu) = {l(s,mu), l(s+mu,nu), l(s+nu,mu), l(s,nu)}
  (Sec. 2.1: one qubit per link, N_l = d L^d, N_p = N_l (d-1)/2, periodic)
* star(s) = {l(s,mu), l(s-mu,mu) for all mu}   (Gauss law G_s, Sec. 2.1)
* W_mu: sigma^z along the non-contractible line of mu-links through the origin
* V_mu: sigma^x on every mu-link of the plane x_mu = 0 (a 't Hooft operator
  pierced by the dual surface); V_mu anticommutes with W_mu, commutes with
  every plaquette and star (Sec. 2.1, eq. for W_mu V_nu).
"""

from __future__ import annotations

import numpy as np


class Lattice:
    def __init__(self, d: int, L):
        L = tuple(int(v) for v in L)
        if d not in (2, 3) or len(L) != d or min(L) < 2:
            raise ValueError("need d in {2,3} and every L_mu >= 2")
        self.d = d
        self.L = L
        self.n_sites = int(np.prod(L))
        self.n_links = d * self.n_sites
        self.plaq_links = []
        self.plaq_planes = []
        for s in range(self.n_sites):
            for mu in range(d):
                for nu in range(mu + 1, d):
                    self.plaq_links.append(self._plaquette(s, mu, nu))
                    self.plaq_planes.append((s, mu, nu))
        self.n_plaq = len(self.plaq_links)
        self.star_links = []
        for s in range(self.n_sites):
            ls = []
            for mu in range(d):
                ls.append(self.link(s, mu))
                ls.append(self.link(self.shift(s, mu, -1), mu))
            self.star_links.append(tuple(ls))

    # -- geometry -----------------------------------------------------------
    def coords(self, s):
        c = []
        for mu in range(self.d):
            c.append(s % self.L[mu])
            s //= self.L[mu]
        return c

    def site(self, c):
        s = 0
        for mu in reversed(range(self.d)):
            s = s * self.L[mu] + (c[mu] % self.L[mu])
        return s

    def shift(self, s, mu, step):
        c = self.coords(s)
        c[mu] += step
        return self.site(c)

    def link(self, s, mu):
        return self.d * s + mu

    def _plaquette(self, s, mu, nu):
        return (
            self.link(s, mu),
            self.link(self.shift(s, mu, 1), nu),
            self.link(self.shift(s, nu, 1), mu),
            self.link(s, nu),
        )

    def plaquette_index(self, s, mu, nu):
        return self.plaq_planes.index((s, mu, nu))

    # -- masks --------------------------------------------------------------
    @staticmethod
    def mask_of(links):
        m = 0
        for l in links:
            m ^= 1 << int(l)
        return m

    def plaq_masks(self):
        return np.array([self.mask_of(p) for p in self.plaq_links], dtype=np.uint64)

    def star_masks(self):
        return np.array([self.mask_of(s) for s in self.star_links], dtype=np.uint64)

    def w_masks(self):
        out = []
        for mu in range(self.d):
            links = [self.link(self.site([n if a == mu else 0 for a in range(self.d)]), mu)
                     for n in range(self.L[mu])]
            out.append(self.mask_of(links))
        return np.array(out, dtype=np.uint64)

    def v_masks(self):
        out = []
        for mu in range(self.d):
            links = [self.link(s, mu) for s in range(self.n_sites) if self.coords(s)[mu] == 0]
            out.append(self.mask_of(links))
        return np.array(out, dtype=np.uint64)

    def area_mask(self, plaquettes):
        """Wilson loop around a set of plaquettes = XOR of their masks."""
        m = 0
        for p in plaquettes:
            m ^= self.mask_of(self.plaq_links[p])
        return m

    def wilson_2x2(self):
        """(mask, degenerate) for the 2x2 loop at the origin in the xy plane.
        A proper contractible 2x2 loop needs L_x, L_y >= 3; otherwise the XOR
        wraps around the torus and the result is flagged degenerate."""
        ps = [self.plaquette_index(self.site([x, y] + [0] * (self.d - 2)), 0, 1)
              for x in (0, 1) for y in (0, 1)]
        m = self.area_mask(ps)
        degenerate = self.L[0] < 3 or self.L[1] < 3
        return m, degenerate

    def contours(self):
        """Contours c1, c2, c3 with perimeters 4:6:8 and areas 1:2:3 (Sec. 3.1);
        the shapes themselves are only in the paper's missing figures.
        2D: plaquette, 1x2 rectangle, L-tromino.  3D (L = 2): plaquette, two
        plaquettes in different planes sharing a link, a 'U' of three."""
        o = 0
        if self.d == 2:
            x1 = self.site([1, 0])
            y1 = self.site([0, 1])
            p0 = self.plaquette_index(o, 0, 1)
            c1 = [p0]
            c2 = [p0, self.plaquette_index(x1, 0, 1)]
            c3 = [p0, self.plaquette_index(x1, 0, 1), self.plaquette_index(y1, 0, 1)]
            deg = [False, self.L[0] < 3, self.L[0] < 3 or self.L[1] < 3]
        else:
            z1 = self.site([0, 0, 1])
            c1 = [self.plaquette_index(o, 0, 1)]
            c2 = [self.plaquette_index(o, 0, 1), self.plaquette_index(o, 0, 2)]
            c3 = [self.plaquette_index(o, 0, 1), self.plaquette_index(o, 0, 2),
                  self.plaquette_index(z1, 0, 1)]
            deg = [False, False, False]
        return [(self.area_mask(c), d_) for c, d_ in zip((c1, c2, c3), deg)]

    def paper_link_number(self, l):
        """1-based link number of the paper's 2D 3x3 figure (Fig. 1b) for our
        link l: the paper counts the +y link of a site before its +x link."""
        if self.d != 2:
            raise ValueError("the paper's numbering is recoverable for d = 2 only")
        s, mu = divmod(int(l), 2)
        return 2 * s + (1 - mu) + 1
