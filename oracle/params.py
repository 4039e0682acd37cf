"""Parameters of the GCA-H^2 construction (oracle side).

The paper fixes the admissibility parameter eta (Sect. 2), the use of a
quadrature rule on the boundary of a box omega around each cluster (Sect. 2),
cross approximation with a reliable (here: complete) pivoting strategy
(Sect. 3), and Sauter's rules for touching triangles (Sect. 8).  It does not
fix the quadrature orders, the ACA stopping rule or the size of omega; the
readings used here are:

* ``omega_margin``: omega = box(tau) widened by omega_margin * diam(tau) on
  every side; default 1/(4 eta), which keeps every admissible partner box
  outside omega (its corners are at most sqrt(3) * margin * diam(tau) away
  from tau, less than the admissible distance diam(tau) / (2 eta)).
* ``aca_tol``: stop before a pivot whose modulus is <= aca_tol times the
  modulus of the first pivot, or when the rank reaches min(rows, 2k).
* ``tie_rel``: pivot candidates within a relative 2^-40 of the maximum
  modulus are treated as tied; the tie goes to the smallest column index,
  then the smallest row index.
* ``sauter_q``: Gauss-Legendre order per variable of the Sauter-Schwab
  rules; disjoint triangle pairs use the 7-point rule on both triangles.
"""

from dataclasses import dataclass


@dataclass
class Params:
    leaf_size: int = 32
    eta: float = 2.0
    box_gauss_m: int = 3
    aca_tol: float = 1e-6
    sauter_q: int = 5
    omega_margin: float = -1.0  # < 0 selects the default 1 / (4 eta)
    tie_rel: float = 2.0 ** -40

    def margin(self):
        if self.omega_margin < 0.0:
            return 1.0 / (4.0 * self.eta)
        return self.omega_margin

    @property
    def k(self):
        """Number of quadrature points on the boundary of omega: 6 m^2."""
        return 6 * self.box_gauss_m * self.box_gauss_m


# The two named build configurations.
SMALL = Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
LARGE = Params(leaf_size=64, eta=2.0, box_gauss_m=4, aca_tol=1e-8, sauter_q=5)
