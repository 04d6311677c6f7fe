"""Writes paper_closed_forms.txt: the exact solutions the paper states for its
accuracy tests, evaluated at m = 8.  Uses only those formulas (no oracle).

  complex   (Sec. 2.1): f_k = F e^{ik}, g_k = G e^{ik}, F = sqrt3 + i sqrt7,
                        G = sqrt5 + i sqrt11, H_k = F G (k+1) e^{ik}
  Hermitian (Sec. 2.3): F = sqrt3, G = sqrt5, H_k = F G (2m-1-k) e^{ik}
"""
import cmath
import math
import os

m = 8
F = complex(math.sqrt(3), math.sqrt(7))
G = complex(math.sqrt(5), math.sqrt(11))
lines = ["# kind k re(H_k) im(H_k); m = 8; see make_closed_forms.py for the cited formulas"]
for k in range(m):
    H = F * G * (k + 1) * cmath.exp(1j * k)
    lines.append(f"complex {k} {H.real!r} {H.imag!r}")
for k in range(m):
    H = math.sqrt(3) * math.sqrt(5) * (2 * m - 1 - k) * cmath.exp(1j * k)
    lines.append(f"hermitian {k} {H.real!r} {H.imag!r}")
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_closed_forms.txt"), "w") as fh:
    fh.write("\n".join(lines) + "\n")
