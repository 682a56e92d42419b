"""GB300-native shared-Jacobian FNLH linear relaxation (arXiv 2404.01407).

The compute path is the CUDA library ``libfnlh.so`` (``csrc/``), reached
through the ctypes binding in :mod:`paper_2404_01407_gb300.fnlh`; this
package's ``__init__`` stays free of it so that :mod:`.inputs` can be
imported without a GPU.
"""

__all__ = ["inputs"]
