"""FP64 CPU oracle for the moment-only ("lightweight") lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run anything here.  The
library in ``paper_2301_01622_gb300`` never imports it, and this package
imports nothing from the library: the two share no code, tables or
constants.

Every function follows a passage of the paper (Tiribocchi et al.,
"Lightweight Lattice Boltzmann", arXiv 2301.01622) and cites it by section
and equation:

* ``lattice``      -- D3Q19 / D3Q27 tables, c_s^2 = 1/3 (Sec. II, III A).
* ``lb``           -- reconstruction (Eqs. (4)-(6)), projection
                      (Eqs. (1)-(3)), collision (Eqs. (7), (8)), pull streaming
                      (Eq. (9)); the moment-only stepper and the two
                      population-storing steppers it is compared with.
* ``diagnostics``  -- mass / momentum sums, <rho>_{rho>0.5} (Sec. IV,
                      Fig. 2), the local relative error of Fig. 3.
* ``two_component``-- colour-gradient two-component model with the
                      near-contact force (Sec. III A-B), in moment-only and
                      population-storing form.

Pins (what each function is checked against, other than itself) are in
``tests/test_oracle_*.py``.
"""
from .lattice import CS2, D3Q19, D3Q27, Lattice, lattice, make_lattice  # noqa: F401
from . import lb, diagnostics  # noqa: F401
