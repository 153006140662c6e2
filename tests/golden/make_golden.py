"""Writes the stored expected values under tests/golden/.

healpix_cap_counts.json: pixel counts of RING polar caps from the ring-size closed
forms of Gorski et al. 2005 (Sect. 4: ring i < nside holds 4 i pixels at
z = 1 - i^2/(3 nside^2); equatorial rings hold 4 nside pixels at
z = 4/3 - 2 i/(3 nside)). Computed here from those integer formulas alone.
"""
import json
import math
import os


def cap_count_closed_form(nside, cap_deg):
    zmin = math.cos(math.radians(cap_deg)) - 1e-12
    total = 0
    for i in range(1, 4 * nside):
        if i < nside:
            z, n = 1.0 - i * i / (3.0 * nside * nside), 4 * i
        elif i <= 3 * nside:
            z, n = 4.0 / 3.0 - 2.0 * i / (3.0 * nside), 4 * nside
        else:
            break
        if z < zmin:
            break
        total += n
    return total


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    cases = [(32, 45.0), (256, 30.0), (1024, 40.0), (4096, 90.0), (1, 90.0), (7, 60.0)]
    out = {"source": "Gorski et al. 2005 ring sizes (the HEALPix tessellation the paper cites in Sect. 1)",
           "cases": [{"nside": n, "cap_deg": d, "count": cap_count_closed_form(n, d)} for n, d in cases]}
    with open(os.path.join(here, "healpix_cap_counts.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
