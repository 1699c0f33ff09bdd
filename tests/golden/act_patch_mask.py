"""Writes act_patch_mask.json: the pixel mask (reading R4 of the oracle: unit-weight
hit block with reciprocal condition >= 1e-3) of the full ACT-like patch, 1024
detectors x 2^20 samples on the 1200x900 TQU map (gen.act_patch(), realisation 0),
computed by the FP64 oracle alone.  The full-size parity test uses it so that the
oracle can evaluate a few detectors of the full operator without re-running the
hit count of all 1024 (about four minutes of CPU).

    python tests/golden/act_patch_mask.py
"""
import base64
import json
import os
import sys
import zlib

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gen  # noqa: E402
from oracle import mapmaker as om  # noqa: E402

OUT = os.path.join(HERE, "act_patch_mask.json")


def main():
    scan, _ = gen.act_patch()
    mask = om.pixel_mask(scan)
    packed = zlib.compress(np.packbits(mask.astype(np.uint8)).tobytes(), 9)
    doc = {
        "what": "pixel mask (R4) of gen.act_patch() realisation 0: 1024 detectors x 2^20 samples, "
                "1200x900 TQU; 1 = kept",
        "cite": "Eq. 3-5 (hit blocks), Eq. 7 (Sigma needs invertible blocks); reading R4",
        "written_by": "python tests/golden/act_patch_mask.py (FP64 oracle only)",
        "ny": scan.ny, "nx": scan.nx, "n_good": int(mask.sum()),
        "packbits_zlib_base64": base64.b64encode(packed).decode(),
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print(f"{OUT}: {int(mask.sum())} of {mask.size} pixels kept, {len(packed)} bytes compressed")


def load():
    """The stored mask as a bool array [ny * nx]."""
    with open(OUT) as f:
        doc = json.load(f)
    bits = np.frombuffer(zlib.decompress(base64.b64decode(doc["packbits_zlib_base64"])), np.uint8)
    return np.unpackbits(bits)[: doc["ny"] * doc["nx"]].astype(bool), doc


if __name__ == "__main__":
    main()
