"""GB300-native (sm_103a) solver of the porosity-extended Saint-Venant model on a
hexagonal raster (arxiv 2406.14933), behind the C ABI of ``include/asx.h``.

``asx``     ctypes binding with the C names (argument marshalling only)
``raster``  a handle built from a synthetic scenario
``inputs``  seeded synthetic terrains, porosity maps and storms
``build``   in-tree nvcc build of ``libasx.so``
"""
from . import inputs  # noqa: F401
