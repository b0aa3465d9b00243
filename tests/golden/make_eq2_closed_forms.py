"""Write eq2_closed_forms.json: closed-form values of the paper's Eq. 2.

Eq. 2 (Sec. 2.1): w = exp[k_normal (d_normal - 1) + k_inplane (d_inplane - 1)]
with the paper's constants k_normal = 10, k_inplane = 5 and thresholds of 25
(normal) and 15 (in-plane) degrees.  Each case fixes d_normal and d_inplane by
a rotation whose dot products are known exactly (Eq. 1).
"""
import json
import math
import os

K_N, K_I = 10.0, 5.0


def eq2(dn, di):
    return math.exp(K_N * (dn - 1.0) + K_I * (di - 1.0))


c10, c20 = math.cos(math.radians(10)), math.cos(math.radians(20))
cases = {
    "source": "Eq. 2 and its constants (k_normal=10, k_inplane=5, thresholds 25/15 deg), Sec. 2.1",
    # rotation by 10 deg about the image normal: beam and lateral both turn by 10 deg
    "tilt10_about_elevation_beam_reading": eq2(c10, c10),
    # same rotation when Eq. 1's normal is read as the image-plane normal: d_normal = 1
    "tilt10_about_elevation_elevation_reading": eq2(1.0, c10),
    # rotation by 20 deg about the lateral axis: only the beam turns
    "tilt20_about_lateral_beam_reading": eq2(c20, 1.0),
    # d_normal = cos 25, d_inplane = cos 15: both thresholds at once
    "both_thresholds": eq2(math.cos(math.radians(25)), math.cos(math.radians(15))),
}
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "eq2_closed_forms.json"), "w") as fh:
    json.dump(cases, fh, indent=1)
    fh.write("\n")
