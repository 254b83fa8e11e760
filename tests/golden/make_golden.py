"""Writes the stored expected values under tests/golden/ from closed forms (no oracle or
GPU code is involved).  Run: python tests/golden/make_golden.py

fig1_parabolic_carving.json -- the worked example of Sec. II, Fig. 1 (caption): parabolic
dispersion eps(k) = |k|^2, q = (0.15, 0, 0), k_F = 0.77.  The doubly carved region of the
method, {eps(k) < eps_F, eps(k + q) > eps_F} with eps_F = k_F^2, is the Fermi ball minus its
overlap with the ball shifted by -q: volume = 4/3 pi R^3 - pi (4R + d)(2R - d)^2 / 12 for two
balls of radius R = k_F whose centres are d = |q| apart (the lens formula)."""
import json
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def lens_volume(R: float, d: float) -> float:
    """Volume of the intersection of two balls of radius R with centres d apart (d <= 2R)."""
    return math.pi * (4.0 * R + d) * (2.0 * R - d) ** 2 / 12.0


def main():
    kF, q = 0.77, (0.15, 0.0, 0.0)
    d = math.sqrt(sum(x * x for x in q))
    ball = 4.0 / 3.0 * math.pi * kF ** 3
    out = {
        "source": "Sec. II, Fig. 1 caption: eps(k) = |k|^2, q = (0.15, 0, 0), k_F = 0.77",
        "kF": kF,
        "q": list(q),
        "ball_volume": ball,
        "carved_volume": ball - lens_volume(kF, d),
        "formula": "4/3 pi kF^3 - pi (4 kF + |q|)(2 kF - |q|)^2 / 12",
    }
    with open(os.path.join(HERE, "fig1_parabolic_carving.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
