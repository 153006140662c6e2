"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and the
benchmark. This package holds geometry and random draws only: none of the
transform's arithmetic lives here."""
from . import configs, healpix, layouts  # noqa: F401
