"""GB300-native IB-GM time step (Wiens & Stockie, arxiv 1305.3976)."""
