"""Run the pass kernels of the checked build on small ragged cases (test helper).

Started by tests/test_gpu_checked.py as a separate process with SNLM_LIBRARY naming
libsnlm_checked.so (built with -DSNLM_CHECKED: guard words after every warp's
shared-memory rows, written before a unit's first store and verified after its
last). Prints one JSON list: per case, the device-side failure record read after
it (snlm_device_error) and the max-abs difference from the FP64 oracle.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from paper_1407_2343_gb300 import _lib, api, synth  # noqa: E402
from paper_1407_2343_gb300.batch import Batch  # noqa: E402

CASES = [
    # H, W, dtype, S, K, profile, order
    (37, 53, "u8", 20, 5, "box", "SURE"),
    (1, 1, "f32", 3, 2, "box", "SURE"),
    (130, 257, "f16", 10, 3, "gauss", "AVG"),
    (9, 300, "u8", 40, 7, "box", "SURE"),        # K = 7 (3 CTAs per SM), lines shorter than a window
    (260, 7, "f32", 6, 0, "box", "CR"),
    (64, 96, "u8", 0, 4, "gauss", "RC"),
    (100, 90, "f32", 33, 6, "gauss", "SURE"),
    (48, 640, "u8", 128, 1, "box", "RC"),        # the largest S
]


def main():
    lib = _lib.load()
    assert os.path.basename(_lib.LIB_PATH) == "libsnlm_checked.so", _lib.LIB_PATH
    oracle.build()
    out = []
    for H, W, dtype, S, K, prof, order in CASES:
        sigma = 20.0
        beta = max(K / 2.0, 0.5)
        img = synth.noisy_image(H, W, sigma, seed=H + W + S, dtype=dtype)
        h = oracle.default_h(sigma, K, prof, beta)
        got = api.snlm_denoise(torch.from_numpy(img).cuda(), S, K, h, prof, order, sigma, beta).cpu().numpy()
        err = api.snlm_device_error()
        ref, _ = oracle.snlm(img.astype(np.float64), S, K, h, prof, beta, order=order, sigma=sigma)
        out.append({"case": f"denoise {H}x{W} {dtype} S={S} K={K} {prof} {order}", "device_error": err,
                    "max_abs": float(np.abs(got - ref).max())})
    # the batched persistent kernel (process_tile under a tile queue)
    reqs = []
    for i, (H, W, dtype, S, K, order) in enumerate([(64, 90, "u8", 5, 2, "RC"), (33, 500, "f16", 10, 3, "SURE"),
                                                     (200, 180, "u8", 12, 5, "AVG")]):
        img = torch.from_numpy(synth.noisy_image(H, W, 25.0, seed=50 + i, dtype=dtype)).cuda()
        o = torch.full((H, W), float("nan"), device="cuda")
        h = api.snlm_default_h(25.0, K)
        reqs.append(dict(img=img, out=o, S=S, K=K, h=h, profile="box", order=order, sigma=25.0, beta=K / 2.0))
    b = Batch(reqs)
    b.run()
    torch.cuda.synchronize()
    status = b.status()
    b.close()
    err = api.snlm_device_error()
    worst = 0.0
    for r in reqs:
        img = r["img"].cpu().numpy().astype(np.float64)
        ref, _ = oracle.snlm(img, r["S"], r["K"], r["h"], "box", r["beta"], order=r["order"], sigma=25.0)
        worst = max(worst, float(np.abs(r["out"].cpu().numpy() - ref).max()))
    out.append({"case": "batch of 3", "device_error": err, "status": status, "max_abs": worst})
    del lib
    print(json.dumps(out))


if __name__ == "__main__":
    main()
