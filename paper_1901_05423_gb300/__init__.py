"""GB300-native radix tree forests for sampling discrete and piecewise
constant distributions (Binder & Keller, arXiv:1901.05423).

The compute path is the CUDA library ``librtf.so`` (sources in ``csrc/``,
interface in ``include/rtf.h``); ``api`` is its Python binding and
``autograd`` wraps the sampler as a differentiable torch function.  Importing
the package does not load the library; the first call does, and fails loudly
if it cannot.
"""

from .api import (  # noqa: F401
    FOREST_MARGINAL, SAMPLE_1D, SAMPLE_2D, SAMPLE_BSEARCH, SAMPLE_COHERENT, Forest,
    GradientAccumulator, RtfError, check_bounded_wait, get_launch_shape, reset_launch_shape,
    set_launch_shape,
    load_statistics, plan_batched, rtf_build, rtf_build_batched, rtf_build_quad, rtf_sample,
    rtf_sample_backward, rtf_sample_loads, rtf_sample_pipelined, rtf_sample_quad, u32_tensor,
)
