"""GB300-native ISRS GN integral model (arXiv 2401.18022).

``workloads`` builds seeded synthetic scenarios; ``api.Engine`` drives the
CUDA library through its C ABI (include/isrs_gn.h).  Importing the package
does not load the library; the first ``api.Engine`` does, and fails loudly
when it is missing or no GPU is present.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "api"]
