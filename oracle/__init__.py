"""FP64 CPU oracle of the S3TTV P-PDS solver.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline /
reference arm may import, call or execute anything under ``oracle/``.  The
product path (``paper_2404_03313_gb300``) never imports it and shares no code with
it; the only module both sides read is ``synthetic`` (seeded inputs, none of the
method's arithmetic).

Every function here is pinned by a ``-m "not gpu"`` test against something other
than itself (brute force on tiny inputs, closed forms, optimality conditions,
invariances, values the paper prints).  See ``oracle/s3ttv.py`` (Alg. 1) and
``oracle/unet.py`` (the network of the learned warm start, which the paper does
not have; import it as ``oracle.unet``).
"""
from .s3ttv import *  # noqa: F401,F403
from .s3ttv import __all__  # noqa: F401
