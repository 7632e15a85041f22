"""GB300-native reconstruction of cut quantum circuits (CutQC post-processing:
attribution, full-definition and dynamic-definition reconstruction) behind a
C ABI (include/cutqc.h).  ``cutqc`` is the thin Python binding."""
from . import cutqc  # noqa: F401
