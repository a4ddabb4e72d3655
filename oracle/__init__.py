"""FP64 CPU oracle for the DPCS path tracer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never calls it;
it shares no code with it.  See ``oracle/dpcs_oracle.c`` for the equations it
follows and the readings it takes where the paper is silent.
"""
from .oracle import (  # noqa: F401
    OrParams,
    OrView,
    build,
    closest,
    lbvh,
    load,
    morton,
    num_threads,
    philox,
    prf,
    render,
    render_backward,
    crf_grad,
    pose_backward,
    bsdf_eval,
    pbr_eval,
    bsdf_pdf,
    bsdf_sample,
    ggx_D,
    adam_step,
    gbuffer,
    denoise,
    denoise_backward,
    l1_loss,
    tv_loss,
)
