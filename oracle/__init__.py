"""FP64 CPU oracle of the SRT3D hot path (test infrastructure).

This package is test infrastructure, not product code: only the test suite,
the smoke check in ``__graft_entry__`` and the CPU-baseline / reference arm of
``bench.py`` may import it. It shares no code with the CUDA path (no kernels,
headers, helpers, tables or constants); its only shared dependency is the
seeded input generator ``paper_2203_00952_gb300.synth``.

Everything is plain numpy in float64, written step by step in the order and
notation of the paper (Sec. 2, Eqs. 1-6; Sec. 3, Eq. 8). The reconstruction
iteration (gradient step, APSS depth denoiser, intensity smoothing) is not
spelled out in the paper, which defers it to RT3D; the oracle fixes one reading
of it, documented in ``oracle.reconstruct``.

Pins (tests that tie the oracle to something other than itself) live in
``tests/test_oracle_pins.py``. Functions with no independent pin say
"parity unpinned" in their docstring.
"""
from .sketch import (  # noqa: F401
    phase_indices,
    sketch_stream,
    sketch_hist,
    hist_from_stream,
    finalize,
    merge_states,
)
from .model import (  # noqa: F401
    h_hat,
    model_cf,
    sketched_loss,
    sketched_gradient,
    sigma_theta,
    weighting_matrix,
    weighted_loss,
    weighted_gradient,
    SIGMA_RIDGE,
)
from .reconstruct import (  # noqa: F401
    Params,
    step_sizes,
    init_matched_filter,
    matched_filter_scores,
    gradient_step,
    neighbour_weights,
    plane_normals,
    apss_depth,
    smooth_prune,
    iterate,
    birth_step,
    reconstruct,
)
