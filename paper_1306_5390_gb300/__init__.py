"""GB300 (sm_103a) implementation of the P-HGRMS salt-and-pepper denoiser.

The method (Algorithms 1-2 and the Section 2 iteration of the paper) runs in
hand-written CUDA kernels behind the C ABI of ``include/hgrms.h``; this
package holds those kernels (``csrc/``), their build (``build.py``), the
ctypes binding (``hgrms.py``) and the seeded synthetic inputs (``synth.py``).
Importing the package loads nothing; the CUDA library is loaded on first use
and its absence raises an error.
"""

__all__ = ["hgrms", "synth", "build"]
