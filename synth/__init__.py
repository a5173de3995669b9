"""Seeded synthetic inputs (random bits and simulated barrel and endcap events) shared by the CUDA
path's tests and bench and by the oracle's tests.  Holds none of the Kalman-filter
arithmetic of the method."""
from .events import FORWARD_ETA, FORWARD_PRIOR, Detector, EventBatch, EventSpec, concat, event_sizes, forward_detector, generate  # noqa: F401
from .philox import normals, philox4x32_10, uniform53, uniforms  # noqa: F401
