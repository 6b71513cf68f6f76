"""Writes tests/golden/bootstrap_b24.json: digests of the oracle's full-ring bootstrap.

The oracle (oracle/bootstrap.py) bootstraps one seeded level-0 ciphertext at ring 2^16 on the
B24 chain (24 + 6 primes of 50 bits, weight-64 secret): the input's 2^15 slot values are drawn
uniform in [-1, 1] by numpy's default generator with seed 5, encrypted at scale 2^40 with nonce
50.  The file records the SHA-256 of the oracle's output words (coefficient form, [2][l+1][n]
uint64, little-endian), its level and scale, a SHA-256 of the diagonal plaintexts the oracle
encoded (so a test can tell an encoder difference from an arithmetic one), and the first words
of every output limb; the same for the bootstrap with its error bootstrapped and subtracted
(meta_bootstrap, kb = 10).  Only oracle/ is called.  The plaintexts come from numpy's FFT, whose
last bits can differ between builds, so the file is written on the machine whose numpy the GPU
test uses.

    python tests/golden/make_bootstrap_golden.py [out.json]
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bootstrap as B  # noqa: E402
from oracle.ckks import Context  # noqa: E402
from oracle.params import B24  # noqa: E402

SEED_Z, NONCE = 5, 50


def plaintext_digest(ctx, plan):
    h = hashlib.sha256()
    for name, levels in (("cts", plan.cts), ("stc", plan.stc)):
        for i, lv in enumerate(levels):
            pts = plan.plaintexts(ctx, name, i)
            for gi in lv.giants:
                for j in sorted(lv.baby[gi]):
                    h.update(np.ascontiguousarray(pts[(gi, j)], dtype="<i8").tobytes())
    return h.hexdigest()


def main():
    out_path = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                                   "bootstrap_b24.json")
    t0 = time.time()
    ctx = Context(B24)
    plan = B.BootPlan(ctx)
    B.gen_boot_keys(ctx, plan)
    z = np.random.default_rng(SEED_Z).uniform(-1, 1, ctx.N)
    ct = ctx.encrypt(z, 0, 2.0 ** 40, nonce=NONCE)
    pdig = plaintext_digest(ctx, plan)
    out = B.bootstrap(ctx, ct, plan)
    words = np.ascontiguousarray(out.c, dtype="<u8")
    err = float(np.max(np.abs(ctx.decrypt(out) - z)))
    meta = B.meta_bootstrap(ctx, ct, plan, kb=10)
    mwords = np.ascontiguousarray(meta.c, dtype="<u8")
    rec = {
        "what": "oracle bootstrap of one seeded level-0 ciphertext, ring 2^16, B24 chain",
        "params": "B24", "seed_z": SEED_Z, "nonce": NONCE, "input_scale": 2.0 ** 40,
        "out_level": out.level, "out_scale": out.scale,
        "sha256_words": hashlib.sha256(words.tobytes()).hexdigest(),
        "sha256_plaintexts": pdig,
        "first_words": words[:, :, :4].tolist(),
        "max_abs_error": err,
        "meta": {"kb": 10, "out_level": meta.level, "out_scale": meta.scale,
                 "sha256_words": hashlib.sha256(mwords.tobytes()).hexdigest(),
                 "first_words": mwords[:, :, :4].tolist(),
                 "max_abs_error": float(np.max(np.abs(ctx.decrypt(meta) - z)))},
        "numpy": np.__version__,
        "seconds": time.time() - t0,
    }
    with open(out_path, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps({k: rec[k] for k in ("out_level", "sha256_words", "max_abs_error", "seconds")}))


if __name__ == "__main__":
    main()
