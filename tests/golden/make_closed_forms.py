"""Write closed_forms.json: textbook closed forms used as fixed expected values.

Values come from the mathematics alone (no oracle, no CUDA):
  brdf_rough_dielectric_60deg -- Eq. 4 read as Cook-Torrance with GGX D,
    Schlick F and separable Smith-GGX, at roughness 1 (alpha_r = 1, so
    D = 1/pi and the visibility term is 1/((1 + n.wo)(1 + n.wi))), metallic 0
    (F0 = 0.04), w_o = n and w_i at 60 degrees from n (half vector at 30).
  lone_gaussian_alpha -- Eq. 3 with a single Gaussian whose mean sits on the
    pixel centre (p = 0): alpha = o = sigmoid(logit).
"""
import json
import math
import os

out = {}
vh = math.cos(math.pi / 6)
F = 0.04 + 0.96 * (1 - vh) ** 5
out["brdf_rough_dielectric_60deg"] = {
    "cite": "Eq. 4 (Section 3.1, Relightable 3D Gaussians)",
    "n": [0, 0, 1], "wo": [0, 0, 1], "wi": [math.sin(math.pi / 3), 0, 0.5],
    "base": 0.3, "rough": 1.0, "metal": 0.0,
    "fs": (1 / math.pi) * F / ((1 + 1) * (1 + 0.5)),
    "fd": 0.3 / math.pi,
}
out["lone_gaussian_alpha"] = {
    "cite": "Eq. 3 and the alpha definition after it (Section 3.1)",
    "logit": 0.3, "alpha": 1 / (1 + math.exp(-0.3)),
}
path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_forms.json")
with open(path, "w") as fh:
    json.dump(out, fh, indent=1)
print(path)
