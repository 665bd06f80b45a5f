"""Worker side of the full-size plane comparison in test_gpu_large.py: each
worker process computes oracle bin planes of the 8192 x 8192 frame (one
independent run of Algorithm 1 per plane) and returns their SHA-256
digests.  Imports nothing but numpy and the oracle, so spawned workers start
quickly."""
import hashlib

import oracle

_IMG = None


def init(img):
    global _IMG
    _IMG = img


def plane_digest(args):
    nbins, k = args
    ref = oracle.integral_histogram_plane(_IMG, nbins, k)
    return k, hashlib.sha256(ref.tobytes() if not ref.flags.c_contiguous else ref).hexdigest()
