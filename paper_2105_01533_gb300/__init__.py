"""GB300-native sparse-state quantum gate application (arXiv 2105.01533).

The compute path lives in ``libsps.so`` (CUDA for sm_103a behind the C ABI in
``include/sps.h``); :mod:`.sps` is its thin ctypes binding and :mod:`.workloads`
holds the seeded input generators. Importing this package loads nothing; the
library is loaded on first use of :mod:`.sps`.
"""

__all__ = ["sps", "workloads", "build"]
