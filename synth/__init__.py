"""Seeded synthetic inputs shared by the oracle tests and the CUDA path: HEALPix geometry, a
LiteBIRD-like sky simulator, spherical K-means patches and named workloads. No part of the
component-separation method is computed here."""
