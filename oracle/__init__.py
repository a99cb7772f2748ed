"""FP64 CPU oracle of the FNO SA-DSRG-PT2 hot path (arXiv:2312.07008).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by bench.py's CPU-baseline and reference legs, never by the library.  It
shares no code with the CUDA path; both read problems from `synth`.
"""
from .dsrg_pt2 import *  # noqa: F401,F403
