"""GB300-native localized style-transfer loss and image gradient (Galerne et al., arXiv 2212.13459).

The compute path is the C-ABI library ``libnst.so`` (hand-written sm_103a CUDA kernels); this
package holds its thin ctypes binding (``native``), the ``torch.autograd.Function`` wrapper and the
L-BFGS / multiscale driver loop (``driver``), and the seeded input generators (``synth``).
Importing the package does not load the library; the first call does, and fails loudly if the
library has not been built.
"""
__all__ = ["native", "synth"]
